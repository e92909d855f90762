// Far-field map over the rotated contour (eq. (FFmap) with eq. (I2complex)):
//   F(a) = k^2 e^{i d gamma} h^d sum_j P(a, j) g_j,
//   g_j = chi(z_j) (u_in(z_j) + u_j),  P(a, j) = prod_c exp(-i k e^{i gamma} alpha_{a,c} x_{j,c}).
//
// The phase factorises over the axes, so the sum is computed in two stages:
//   stage 1  T[k][rho] = sum_ix P_x(k, ix) g[rho][ix]       (rho = row index (iz, iy))
//   stage 2  F[a]      = sum_rho P_y(a, iy) [P_z(a, iz)] T[xrow(a)][rho]
// where k runs over the distinct x-components of the outgoing directions
// (mirror-image directions share them).  Arithmetic is FP64 throughout.
//
// Range: with a rotated contour |P| grows like e^{k sin(gamma) alpha.x} and
// |g| like e^{k sin(gamma) |x|} at the upstream edge; for large k R the terms
// leave the FP64 range.  Stage 1 folds a power of two 2^-s1 into the x-table
// when an a-priori bound on |T| exceeds 2^1020, stage 2 picks 2^-s2 from the
// largest term of its own sum; the result is returned as F' with exponent
// s1 + s2 (F = F' 2^(s1+s2)).
#include <cmath>
#include <map>
#include <vector>

#include "csff_internal.h"

namespace csff {
namespace {

__device__ __forceinline__ int exp2_of(double a) {
  if (a == 0.0) return -4000;
  int e;
  frexp(a, &e);
  return e;
}

__device__ __forceinline__ int cexp2(double2 v) { return exp2_of(fmax(fabs(v.x), fabs(v.y))) + 1; }

// g = chi (u_in + u) at every interior node.
struct Tabs8 { const double2* p[8]; };

template <int D>
__global__ void k_gfield(Tabs8 tabs, int n_gauss, const double2* __restrict__ uinc,
                         const double2* __restrict__ u, int m, double2* __restrict__ g) {
  int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y;
  int iz = (D == 3) ? (int)blockIdx.z : 0;
  if (ix >= m || iy >= m) return;
  long long idx = ((long long)iz * m + iy) * m + ix;
  // g = chi u_in + chi u; chi u_in with each axis' Gaussian factor paired with
  // its incident-wave factor first (no partial product beyond the FP64 range)
  double2 chi = make_double2(0, 0), cu = make_double2(0, 0);
  for (int q = 0; q < n_gauss; ++q) {
    const double2* t = tabs.p[q];
    double2 v = cmul(t[ix], t[m + iy]);
    double2 w = cmul(cmul(t[ix], uinc[ix]), cmul(t[m + iy], uinc[m + iy]));
    if (D == 3) {
      v = cmul(v, t[2 * m + iz]);
      w = cmul(w, cmul(t[2 * m + iz], uinc[2 * m + iz]));
    }
    chi = cadd(chi, v);
    cu = cadd(cu, w);
  }
  g[idx] = cadd(cu, cmul(chi, u[idx]));
}

// Phase tables.  x-table rows k < n_ux: P_x(k, i) 2^-s1[k]; y/z tables for
// every angle: ytab[a][i], ztab[a][i] (unscaled).  x_i = lo + (i + 1) h.
// s1[k] = max(0, bound_exp(P_x row) + gmax + ceil(log2 m) + 2 - 1020).
__global__ void k_phase_tables(const double* __restrict__ ux, int n_ux, const double* __restrict__ alpha,
                               int n_ang, int dim, int m, double lo, double h, double k, double sg,
                               double cg, const int* __restrict__ gmax, double2* __restrict__ xtab,
                               double2* __restrict__ ytab, double2* __restrict__ ztab,
                               int* __restrict__ s1, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int row = blockIdx.y;
  if (i >= m) return;
  const double LN2 = 0.69314718055994530942;
  double x = lo + (double)(i + 1) * h;
  if (row < n_ux) {
    double a = ux[row];
    double xmax = fmax(a * (lo + h), a * (lo + (double)m * h));   // max_i a x_i
    int bx = (int)ceil(k * sg * xmax / LN2) + 1;
    int lm = 0;
    while ((1 << lm) < m) ++lm;
    int s = bx + *gmax + lm + 2 - 1020;
    s = s > 0 ? s : 0;
    if (i == 0) { s1[row] = s; if (s > 0) atomicOr(flag, 1); }
    double mag = exp(k * sg * a * x - (double)s * LN2);
    double sn, cs;
    sincos(k * cg * a * x, &sn, &cs);
    xtab[(long long)row * m + i] = make_double2(mag * cs, -mag * sn);
  } else {
    int ar = row - n_ux;                 // y (and z) tables for angle ar
    if (ar >= n_ang) return;
    for (int c = 1; c < dim; ++c) {
      double a = alpha[(long long)ar * dim + c];
      double mag = exp(k * sg * a * x);
      double sn, cs;
      sincos(k * cg * a * x, &sn, &cs);
      double2 v = make_double2(mag * cs, -mag * sn);
      if (c == 1) ytab[(long long)ar * m + i] = v;
      else ztab[(long long)ar * m + i] = v;
    }
  }
}

// Stage 1: T[k][rho] = sum_i X[k][i] G[rho][i]   (complex, FP64).
// FP64 FMA throughput (about 2 per SM per clock) bounds this kernel, so the
// tiles are small (16 rows x 32 columns, K step 16; 2 outputs per thread) to
// give several CTAs per SM and a short last wave.
constexpr int S1_BM = 16, S1_BN = 32, S1_BK = 16;

// Choice between the two stage-1 kernels, taken on the device from the block
// spreads (max - min exponent inside one block of one row) of the two operands.
// With x' = 2^-ex x and g' = 2^-eg g every block holds a node where |x'| >= 1/2
// and one where |g'| >= 1/2, so the largest scaled product of a block is at
// least 2^-(min(sx, sg) + 2); products flushed below FP32's subnormal range
// (2^-149) then cost at most 2^-149 * DKB absolute, far under the double-float
// rounding (2^-47 relative) of that largest product when min(sx, sg) <= 90.
constexpr int DF_SPREAD_LIMIT = 90;       // bits
constexpr int DF_NONFINITE = 100000;      // spread written for a block with a NaN/Inf
__device__ __forceinline__ bool df_selected(const int* __restrict__ spread) {
  const int sx = spread[0], sg = spread[1];
  return sx < DF_NONFINITE && sg < DF_NONFINITE && min(sx, sg) <= DF_SPREAD_LIMIT;
}

__global__ void __launch_bounds__(256) k_ff_stage1(const double2* __restrict__ X, int M,
                                                   const double2* __restrict__ G, int N, int K,
                                                   double2* __restrict__ T, const int* __restrict__ skip_if_df) {
  if (skip_if_df && df_selected(skip_if_df)) return;   // the double-float kernel ran
  __shared__ double2 As[S1_BK][S1_BM];
  __shared__ double2 Bs[S1_BK][S1_BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;     // tx: column pair, ty: row
  const int m0 = blockIdx.y * S1_BM, n0 = blockIdx.x * S1_BN;
  double2 acc0 = make_double2(0, 0), acc1 = make_double2(0, 0);
  for (int k0 = 0; k0 < K; k0 += S1_BK) {
    {                                        // A tile: 16 x 16
      int r = tid >> 4, kk = tid & 15;
      int gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < K) ? X[(long long)gm * K + gk] : make_double2(0, 0);
    }
#pragma unroll
    for (int l = 0; l < 2; ++l) {            // B tile: 32 x 16
      int e = tid + l * 256;
      int r = e >> 4, kk = e & 15;
      int gn = n0 + r, gk = k0 + kk;
      Bs[kk][r] = (gn < N && gk < K) ? G[(long long)gn * K + gk] : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < S1_BK; ++kk) {
      double2 a = As[kk][ty];
      double2 b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      acc0.x = fma(a.x, b0.x, fma(-a.y, b0.y, acc0.x));
      acc0.y = fma(a.x, b0.y, fma(a.y, b0.x, acc0.y));
      acc1.x = fma(a.x, b1.x, fma(-a.y, b1.y, acc1.x));
      acc1.y = fma(a.x, b1.y, fma(a.y, b1.x, acc1.y));
    }
    __syncthreads();
  }
  int gm = m0 + ty;
  if (gm < M) {
    int gn = n0 + tx * 2;
    if (gn < N) T[(long long)gm * N + gn] = acc0;
    if (gn + 1 < N) T[(long long)gm * N + gn + 1] = acc1;
  }
}

template <typename V, typename Op>
__device__ __forceinline__ V bred(V v, Op op, V* sh) {
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = sh[0];
  for (int j = 1; j < (int)(blockDim.x >> 5); ++j) v = op(v, sh[j]);
  return v;
}
struct MaxI { __device__ int operator()(int a, int b) const { return a > b ? a : b; } };
struct AddD { __device__ double operator()(double a, double b) const { return a + b; } };

// Stage 2: one block per angle.
template <int D>
__global__ void k_ff_stage2(const double2* __restrict__ T, const int* __restrict__ xrow,
                            const int* __restrict__ s1, const double2* __restrict__ ytab,
                            const double2* __restrict__ ztab, int m, double2 pref,
                            double2* __restrict__ F, int* __restrict__ Fexp, int write_exp,
                            int* __restrict__ flag) {
  __shared__ int shi[32];
  __shared__ double shd[32];
  const int a = blockIdx.x;
  const int kx = xrow[a];
  const long long R = (D == 3) ? (long long)m * m : m;
  const double2* Tr = T + (long long)kx * R;
  const double2* yr = ytab + (long long)a * m;
  const double2* zr = ztab + (long long)a * m;
  int emax = -4000;
  for (long long r = threadIdx.x; r < R; r += blockDim.x) {
    int iy = (int)(r % m), iz = (int)(r / m);
    int e = cexp2(Tr[r]) + cexp2(yr[iy]) + ((D == 3) ? cexp2(zr[iz]) : 0);
    emax = e > emax ? e : emax;
  }
  emax = bred(emax, MaxI(), shi);
  int lr = 0;
  while ((1ll << lr) < R) ++lr;
  int s2 = emax + lr + 2 - 1020;
  s2 = s2 > 0 ? s2 : 0;
  double sc = ldexp(1.0, -s2);
  double ax = 0, ay = 0;
  for (long long r = threadIdx.x; r < R; r += blockDim.x) {
    int iy = (int)(r % m), iz = (int)(r / m);
    double2 w = cscale(yr[iy], sc);
    if (D == 3) w = cmul(w, zr[iz]);
    double2 t = Tr[r];
    ax = fma(w.x, t.x, fma(-w.y, t.y, ax));
    ay = fma(w.x, t.y, fma(w.y, t.x, ay));
  }
  ax = bred(ax, AddD(), shd);
  ay = bred(ay, AddD(), shd);
  if (threadIdx.x == 0) {
    double2 f = cmul(pref, make_double2(ax, ay));
    int e = s1[kx] + s2;
    if (s2 > 0) atomicOr(flag, 1);
    if (write_exp) {
      F[a] = f;
      Fexp[a] = e;
    } else {
      F[a] = make_double2(ldexp(f.x, e), ldexp(f.y, e));
    }
  }
}

// ---- stage 1 in double-float arithmetic -------------------------------------
// FP64 runs at 1/61 of the FP32 rate on this part, so stage 1 can also run in
// double-float arithmetic (value = hi + lo, two FP32 numbers, ~48-bit
// significand) on the FP32 pipes: products by Dekker's splitting with FMA
// (TwoProd), sums by Knuth's TwoSum.  Both operands are cut into blocks of
// DKB consecutive x-nodes; inside a block every row of P_x and every row of g
// is scaled by a power of two (ex, eg: exponent of the block maximum), so all
// block sums (|.| <= 2 DKB) are formed in double-float and merged into a
// running double-float sum that carries its own power-of-two exponent:
//   T[k][rho] = sum_b 2^(ex[k][b] + eg[rho][b]) sum_{i in b} P'_x(k, i) g'[rho][i].
// The kernel runs only when df_selected() holds for the measured spreads,
// else the FP64 kernel does.
constexpr int DKB = 32;

struct df { float hi, lo; };

// split x (|x| <= 2) into hi + lo
__device__ __forceinline__ df df_of(double x) {
  float h = (float)x;
  return df{h, (float)(x - (double)h)};
}

// s += a * b  (double-float; s kept unnormalised: hi via TwoSum, lo collects errors)
__device__ __forceinline__ void df_mac(df& s, df a, df b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);          // exact error of the leading product
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float t = s.hi + p;                      // TwoSum(s.hi, p)
  float v = t - s.hi;
  float err = (s.hi - (t - v)) + (p - v);
  s.hi = t;
  s.lo += err + e;
}

__device__ __forceinline__ int ilog2_up(double a) {   // exponent e with a < 2^e (a > 0)
  int e;
  frexp(a, &e);
  return e;
}

// one warp per (row, block): block exponent of |v| (upper bound), scaled
// double-float split, and the row-block spread (max - min exponent) into *spread
__global__ void k_split_rows(const double2* __restrict__ v, int m, int nrows, float4* __restrict__ vdf,
                             int* __restrict__ ev, int* __restrict__ spread) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nb = (m + DKB - 1) / DKB;
  if (warp >= nrows * nb) return;
  const int row = warp / nb, b = warp % nb;
  const int i = b * DKB + lane;
  double2 x = (i < m) ? v[(long long)row * m + i] : make_double2(0, 0);
  double a = fmax(fabs(x.x), fabs(x.y));
  int e = (a > 0.0 && isfinite(a)) ? ilog2_up(a) : -100000;
  int emin = (a > 0.0 && isfinite(a)) ? e : 100000;
  for (int o = 16; o > 0; o >>= 1) {
    e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
  }
  const bool bad = __any_sync(0xffffffffu, !isfinite(a));   // non-finite: the FP64 kernel runs
  const int eb = (e == -100000 || bad) ? 0 : e;
  if (lane == 0) {
    ev[(long long)row * nb + b] = eb;
    int sp = bad ? DF_NONFINITE : ((e == -100000) ? 0 : e - emin);
    atomicMax(spread, sp);
  }
  // ldexp on the value itself: 2^-eb alone overflows for subnormal blocks
  const bool zero = e == -100000 || bad;
  df re = df_of(zero ? 0.0 : ldexp(x.x, -eb)), im = df_of(zero ? 0.0 : ldexp(x.y, -eb));
  vdf[(long long)row * nb * DKB + b * DKB + lane] = make_float4(re.hi, re.lo, im.hi, im.lo);
}

// 2^d as a float for d <= 0 (0 below the subnormal range): exact power of two
__device__ __forceinline__ float pow2f_neg(int d) {
  if (d >= -126) return __int_as_float((d + 127) << 23);
  if (d >= -149) return __int_as_float(1 << (d + 149));
  return 0.f;
}

// running double-float sum with its own power-of-two exponent:
// value = (hi + lo) 2^E; merging a block sum s 2^Es rescales the smaller of the
// two exactly (powers of two) and adds with TwoSum, all in FP32
struct dfacc { float hi, lo; int E; };

__device__ __forceinline__ void dfacc_merge2(dfacc& re, dfacc& im, df sr, df si, int Es) {
  if (sr.hi == 0.f && si.hi == 0.f && sr.lo == 0.f && si.lo == 0.f) return;
  const int En = max(re.E, Es);                    // re.E == im.E always
  const float fa = pow2f_neg(re.E - En), fs = pow2f_neg(Es - En);
  auto add = [&](dfacc& a, df x) {
    float ah = a.hi * fa, al = a.lo * fa, xh = x.hi * fs, xl = x.lo * fs;
    float t = ah + xh, v = t - ah;
    float err = (ah - (t - v)) + (xh - v);
    float lo = al + xl + err;
    float h = t + lo;                              // renormalise (fast TwoSum)
    a.lo = lo - (h - t);
    a.hi = h;
    a.E = En;
  };
  add(re, sr);
  add(im, si);
}

// T[k][rho] over blocks; 16 (k) x 64 (rho) output tile, 1 x 4 outputs per thread
constexpr int DF_BM = 16, DF_BN = 64;

__global__ void __launch_bounds__(256) k_ff_stage1_df(const float4* __restrict__ X, const int* __restrict__ ex, int M,
                                                      const float4* __restrict__ G, const int* __restrict__ eg, int N,
                                                      int nb, const int* __restrict__ spread,
                                                      double2* __restrict__ T) {
  if (!df_selected(spread)) return;      // the FP64 kernel takes this launch
  __shared__ float4 As[DF_BM][DKB + 1];
  __shared__ float4 Bs[DF_BN][DKB + 1];
  __shared__ int eA[DF_BM], eB[DF_BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * DF_BM, n0 = blockIdx.x * DF_BN;
  dfacc accr[4], acci[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    accr[j] = dfacc{0.f, 0.f, -100000};
    acci[j] = dfacc{0.f, 0.f, -100000};
  }
  for (int b = 0; b < nb; ++b) {
    for (int i = tid; i < DF_BM * DKB; i += 256) {
      int r = i / DKB, kk = i % DKB, gm = m0 + r;
      As[r][kk] = (gm < M) ? X[((long long)gm * nb + b) * DKB + kk] : make_float4(0, 0, 0, 0);
    }
    for (int i = tid; i < DF_BN * DKB; i += 256) {
      int r = i / DKB, kk = i % DKB, gn = n0 + r;
      Bs[r][kk] = (gn < N) ? G[((long long)gn * nb + b) * DKB + kk] : make_float4(0, 0, 0, 0);
    }
    if (tid < DF_BM) eA[tid] = (m0 + tid < M) ? ex[(long long)(m0 + tid) * nb + b] : 0;
    if (tid >= 64 && tid < 64 + DF_BN) eB[tid - 64] = (n0 + tid - 64 < N) ? eg[(long long)(n0 + tid - 64) * nb + b] : 0;
    __syncthreads();
    df sr[4], si[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) { sr[j] = df{0.f, 0.f}; si[j] = df{0.f, 0.f}; }
#pragma unroll 2
    for (int kk = 0; kk < DKB; ++kk) {
      float4 a = As[ty][kk];
      df ar{a.x, a.y}, ai{a.z, a.w}, nai{-a.z, -a.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float4 bb = Bs[tx + 16 * j][kk];
        df br{bb.x, bb.y}, bi{bb.z, bb.w};
        df_mac(sr[j], ar, br);
        df_mac(sr[j], nai, bi);
        df_mac(si[j], ar, bi);
        df_mac(si[j], ai, br);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) dfacc_merge2(accr[j], acci[j], sr[j], si[j], eA[ty] + eB[tx + 16 * j]);
    __syncthreads();
  }
  const int gm = m0 + ty;
  if (gm >= M) return;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int gn = n0 + tx + 16 * j;
    if (gn >= N) continue;
    T[(long long)gm * N + gn] = make_double2(ldexp((double)accr[j].hi + (double)accr[j].lo, accr[j].E),
                                             ldexp((double)acci[j].hi + (double)acci[j].lo, acci[j].E));
  }
}

// ---- 3D sum-factorised contraction --------------------------------------------
// stage A: T1[t][col] = sum_iz Pz[t][iz] g[iz][col] for a group of TB distinct
// z-components t (col = iy m + ix); each thread keeps TB sums in registers so
// g is streamed once per group.
template <int TB>
__global__ void __launch_bounds__(256) k_ff3_stageA(const double2* __restrict__ zt, int T, int t0,
                                                    const double2* __restrict__ g, int m, long long ncol,
                                                    double2* __restrict__ T1) {
  __shared__ double2 zs[TB][32];
  const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double2 acc[TB];
#pragma unroll
  for (int t = 0; t < TB; ++t) acc[t] = make_double2(0, 0);
  for (int k0 = 0; k0 < m; k0 += 32) {
    __syncthreads();
    for (int i = threadIdx.x; i < TB * 32; i += blockDim.x) {
      int t = i / 32, kk = i % 32;
      zs[t][kk] = (t0 + t < T && k0 + kk < m) ? zt[(long long)(t0 + t) * m + k0 + kk] : make_double2(0, 0);
    }
    __syncthreads();
    if (col < ncol) {
      const int kend = min(32, m - k0);
      for (int kk = 0; kk < kend; ++kk) {
        double2 gv = g[(long long)(k0 + kk) * ncol + col];
#pragma unroll
        for (int t = 0; t < TB; ++t) {
          double2 z = zs[t][kk];
          acc[t].x = fma(z.x, gv.x, fma(-z.y, gv.y, acc[t].x));
          acc[t].y = fma(z.x, gv.y, fma(z.y, gv.x, acc[t].y));
        }
      }
    }
  }
  if (col >= ncol) return;
#pragma unroll
  for (int t = 0; t < TB; ++t)
    if (t0 + t < T) T1[(long long)(t0 + t) * ncol + col] = acc[t];
}

// stage B: T2[a][ix] = sum_iy Py[a][iy] T1[t(a)][iy m + ix]
__global__ void __launch_bounds__(128) k_ff3_stageB(const double2* __restrict__ yt, const int* __restrict__ trow,
                                                    const double2* __restrict__ T1, int m,
                                                    double2* __restrict__ T2) {
  extern __shared__ double2 ys[];
  const int a = blockIdx.y;
  for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = yt[(long long)a * m + i];
  __syncthreads();
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= m) return;
  const double2* base = T1 + (long long)trow[a] * m * m + ix;
  double2 acc = make_double2(0, 0);
  for (int iy = 0; iy < m; ++iy) {
    double2 y = ys[iy], t = base[(long long)iy * m];
    acc.x = fma(y.x, t.x, fma(-y.y, t.y, acc.x));
    acc.y = fma(y.x, t.y, fma(y.y, t.x, acc.y));
  }
  T2[(long long)a * m + ix] = acc;
}

// per-angle tables for the 3D path: ztab over distinct z-components, y and x
// tables per angle: P_c(a, i) = exp(-i k e^{i gamma} alpha_c x_i)
__global__ void k_phase_tables3(const double* __restrict__ uz, int n_uz, const double* __restrict__ alpha,
                                int n_ang, int m, double lo, double h, double k, double sg, double cg,
                                double2* __restrict__ ztab, double2* __restrict__ ytab, double2* __restrict__ xtab) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int row = blockIdx.y;
  if (i >= m) return;
  double x = lo + (double)(i + 1) * h;
  auto ph = [&](double a) {
    double mag = exp(k * sg * a * x);
    double sn, cs;
    sincos(k * cg * a * x, &sn, &cs);
    return make_double2(mag * cs, -mag * sn);
  };
  if (row < n_uz) {
    ztab[(long long)row * m + i] = ph(uz[row]);
  } else {
    int a = row - n_uz;
    if (a >= n_ang) return;
    ytab[(long long)a * m + i] = ph(alpha[(long long)a * 3 + 1]);
    xtab[(long long)a * m + i] = ph(alpha[(long long)a * 3 + 0]);
  }
}

}  // namespace

static cudaError_t ensure(void** p, size_t& cap, size_t need, csff_plan* P) {
  if (cap >= need && *p) return cudaSuccess;
  if (*p) { cudaFree(*p); P->bytes -= cap; *p = nullptr; cap = 0; }
  cudaError_t e = cudaMalloc(p, need);
  if (e == cudaSuccess) { cap = need; P->bytes += need; }
  return e;
}

void free_ff_buffers(csff_plan* P) {
  FFBuffers& b = P->ff;
  for (void* p : {(void*)b.dg, (void*)b.dxt, (void*)b.dyt, (void*)b.dzt, (void*)b.dT, (void*)b.dal,
                  (void*)b.dux, (void*)b.dxr, (void*)b.ds1, (void*)b.dmisc, (void*)b.dxdf, (void*)b.dgdf,
                  (void*)b.dex, (void*)b.deg, (void*)b.dspread})
    if (p) cudaFree(p);
  b = FFBuffers{};
}

csff_status far_field_one(csff_plan* P, const double* eta_host, const double2* u, int n_ang,
                          const double* alpha_host, double2* F, int32_t* F_exp, bool* scaled) {
  const int d = P->dim;
  const Level& L = P->lv[0];
  const int m = L.m;
  cudaStream_t s = P->stream;
  FFBuffers& B = P->ff;
  cudaError_t e;
  // distinct x-components (bitwise) -> rows of the x-table.  (Pairing +a
  // with -a through even/odd parts of g would halve the work but multiplies
  // e^{+k sin(gamma) a |x|} with the large upstream g; the cross terms exceed
  // the sum by up to e^{2 k sin(gamma) a R}, so the plain form is kept.)
  std::vector<double> ux;
  std::vector<int> xr(n_ang);
  std::map<double, int> seen;
  for (int a = 0; a < n_ang; ++a) {
    double v = alpha_host[(size_t)a * d];
    auto it = seen.find(v);
    if (it == seen.end()) { it = seen.emplace(v, (int)ux.size()).first; ux.push_back(v); }
    xr[a] = it->second;
  }
  const int n_ux = (int)ux.size();
  const int n_trow = n_ux;
  const long long R = (d == 3) ? (long long)m * m : m;
  if ((e = ensure((void**)&B.dg, B.g, sizeof(double2) * (size_t)L.N, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dxt, B.xt, sizeof(double2) * (size_t)n_ux * m, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dyt, B.yt, sizeof(double2) * (size_t)n_ang * m, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dzt, B.zt, sizeof(double2) * (size_t)n_ang * m, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dal, B.al, sizeof(double) * (size_t)n_ang * d, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dux, B.ux, sizeof(double) * (size_t)n_ux, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dxr, B.xr, sizeof(int) * (size_t)n_ang, P)) != cudaSuccess ||
      (e = ensure((void**)&B.ds1, B.s1, sizeof(int) * (size_t)n_trow, P)) != cudaSuccess) {
    return e == cudaErrorMemoryAllocation ? (set_error("far field: device allocation failed"), CSFF_ERR_OOM)
                                          : cuda_fail(e, "far field scratch");
  }
  if (!B.dmisc) {
    if ((e = cudaMalloc((void**)&B.dmisc, 4 * sizeof(int))) != cudaSuccess) return cuda_fail(e, "malloc");
  }
  // incident-wave tables for eta: U_c[i] = exp(i k eta_c z_i)
  {
    std::vector<double2> ut((size_t)d * m);
    const double cg = std::cos(P->prob.gamma), sg = std::sin(P->prob.gamma);
    for (int c = 0; c < d; ++c)
      for (int i = 0; i < m; ++i) {
        double x = P->prob.box_lo + (double)(i + 1) * L.h;
        double t = P->prob.k * eta_host[c] * x;   // i k eta_c x e^{i g} = -k sg t + i k cg t
        double mag = std::exp(-sg * t);
        ut[(size_t)c * m + i] = make_double2(mag * std::cos(cg * t), mag * std::sin(cg * t));
      }
    if ((e = cudaMemcpyAsync(P->uinc_tab, ut.data(), sizeof(double2) * ut.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return cuda_fail(e, "upload incident tables");
  }
  if ((e = cudaMemcpyAsync(B.dal, alpha_host, sizeof(double) * (size_t)n_ang * d, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(B.dux, ux.data(), sizeof(double) * n_ux, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(B.dxr, xr.data(), sizeof(int) * n_ang, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(B.dmisc + 1, 0, sizeof(int), s)) != cudaSuccess)
    return cuda_fail(e, "upload angles");

  Tabs8 t{};
  for (int q = 0; q < P->prob.n_gauss; ++q) t.p[q] = P->chi_tab[0] + (size_t)q * d * m;   // finest level
  dim3 gg((m + 31) / 32, (m + 7) / 8, d == 3 ? m : 1), gb(32, 8);
  if (d == 2) k_gfield<2><<<gg, gb, 0, s>>>(t, P->prob.n_gauss, P->uinc_tab, u, m, B.dg);
  else k_gfield<3><<<gg, gb, 0, s>>>(t, P->prob.n_gauss, P->uinc_tab, u, m, B.dg);
  count_launch();
  if ((e = launch_max_exp(B.dg, L.N, B.dmisc, s)) != cudaSuccess) return cuda_fail(e, "max exponent");
  const double sg = std::sin(P->prob.gamma), cg = std::cos(P->prob.gamma);
  if (d == 3) {
    // sum-factorised path when no intermediate can leave the FP64 range:
    // |T1| <= m max|Pz| max|g|, |T2| <= m max|Py| |T1|, terms of stage C
    // scaled from their own maximum
    int gmax = 0;
    if ((e = cudaMemcpyAsync(&gmax, B.dmisc, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "far field range");
    const double R = std::max(std::fabs(P->prob.box_lo), std::fabs(P->prob.box_hi));
    const double lp = P->prob.k * sg * R / std::log(2.0);
    const double bound = gmax + 2 * lp + 2 * std::log2((double)m) + 4;
    if (bound < 1000.0 && gmax < 2000) {
      std::vector<double> uz;
      std::vector<int> tr(n_ang);
      std::map<double, int> zseen;
      for (int a = 0; a < n_ang; ++a) {
        double v = alpha_host[(size_t)a * 3 + 2];
        auto it = zseen.find(v);
        if (it == zseen.end()) { it = zseen.emplace(v, (int)uz.size()).first; uz.push_back(v); }
        tr[a] = it->second;
      }
      const int n_uz = (int)uz.size();
      const long long ncol = (long long)m * m;
      // scratch: ztab in dxt, y/x tables in dyt/dzt, T1 in dT, T2 after T1, rows in dxr, zero s1
      if ((e = ensure((void**)&B.dxt, B.xt, sizeof(double2) * (size_t)std::max(n_uz, 1) * m, P)) != cudaSuccess ||
          (e = ensure((void**)&B.dT, B.T, sizeof(double2) * ((size_t)n_uz * ncol + (size_t)n_ang * m), P)) !=
              cudaSuccess ||
          (e = ensure((void**)&B.dux, B.ux, sizeof(double) * (size_t)std::max(n_uz, 1), P)) != cudaSuccess ||
          (e = ensure((void**)&B.ds1, B.s1, sizeof(int) * (size_t)n_ang, P)) != cudaSuccess)
        return cuda_fail(e, "far field scratch");
      std::vector<int> ident(n_ang);
      for (int a = 0; a < n_ang; ++a) ident[a] = a;
      if ((e = cudaMemcpyAsync(B.dux, uz.data(), sizeof(double) * n_uz, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
          (e = cudaMemcpyAsync(B.dxr, tr.data(), sizeof(int) * n_ang, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
          (e = cudaMemsetAsync(B.ds1, 0, sizeof(int) * n_ang, s)) != cudaSuccess)
        return cuda_fail(e, "far field tables");
      dim3 tg3((m + 127) / 128, n_uz + n_ang);
      k_phase_tables3<<<tg3, 128, 0, s>>>(B.dux, n_uz, B.dal, n_ang, m, P->prob.box_lo, L.h, P->prob.k, sg, cg,
                                          B.dxt, B.dyt, B.dzt);
      double2* T1 = B.dT;
      double2* T2 = B.dT + (size_t)n_uz * ncol;
      {
        ProfScope ps(PF_FF_CONTRACT, s, 16.0 * ((double)n_uz * m + (double)ncol * m + (double)n_uz * ncol),
                     8.0 * (double)n_uz * (double)ncol * m);
        for (int t0 = 0; t0 < n_uz; t0 += 16)
          k_ff3_stageA<16><<<(unsigned)((ncol + 255) / 256), 256, 0, s>>>(B.dxt, n_uz, t0, B.dg, m, ncol, T1);
      }
      k_ff3_stageB<<<dim3((m + 127) / 128, n_ang), 128, sizeof(double2) * m, s>>>(B.dyt, B.dxr, T1, m, T2);
      // stage C: F[a] = pref sum_ix Px[a][ix] T2[a][ix]  (the 2D stage-2 kernel on rows a)
      if ((e = cudaMemcpyAsync(B.dxr, ident.data(), sizeof(int) * n_ang, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "far field rows");
      const double hd = std::pow(L.h, 3);
      const double k2 = P->prob.k * P->prob.k;
      double2 pref = make_double2(k2 * hd * std::cos(3 * P->prob.gamma), k2 * hd * std::sin(3 * P->prob.gamma));
      k_ff_stage2<2><<<n_ang, 256, 0, s>>>(T2, B.dxr, B.ds1, B.dzt, B.dzt, m, pref, F, F_exp, F_exp != nullptr,
                                           B.dmisc + 1);
      count_launch(3 + (n_uz + 15) / 16);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "far field 3D kernels");
      if (scaled) {
        int flag = 0;
        if ((e = cudaMemcpyAsync(&flag, B.dmisc + 1, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
          return cuda_fail(e, "far field flag");
        *scaled = flag != 0;
      }
      return CSFF_OK;
    }
  }
  if ((e = ensure((void**)&B.dT, B.T, sizeof(double2) * (size_t)n_trow * R, P)) != cudaSuccess)
    return cuda_fail(e, "far field scratch");
  dim3 tg((m + 127) / 128, n_ux + n_ang);
  k_phase_tables<<<tg, 128, 0, s>>>(B.dux, n_ux, B.dal, n_ang, d, m, P->prob.box_lo, L.h, P->prob.k, sg, cg,
                                    B.dmisc, B.dxt, B.dyt, B.dzt, B.ds1, B.dmisc + 1);
  count_launch();
  // operands of the double-float contraction
  const int nbk = (m + DKB - 1) / DKB;
  if ((e = ensure((void**)&B.dxdf, B.xdf, sizeof(float4) * (size_t)n_ux * nbk * DKB, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dgdf, B.gdf, sizeof(float4) * (size_t)R * nbk * DKB, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dex, B.exs, sizeof(int) * (size_t)n_ux * nbk, P)) != cudaSuccess ||
      (e = ensure((void**)&B.deg, B.egs, sizeof(int) * (size_t)R * nbk, P)) != cudaSuccess)
    return cuda_fail(e, "far field scratch");
  if (!B.dspread && (e = cudaMalloc((void**)&B.dspread, 2 * sizeof(int))) != cudaSuccess)
    return cuda_fail(e, "far field scratch");
  if ((e = cudaMemsetAsync(B.dspread, 0, 2 * sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "memset");
  {
    const long long wx = (long long)n_ux * nbk, wg = (long long)R * nbk;
    k_split_rows<<<(unsigned)((wx * 32 + 255) / 256), 256, 0, s>>>(B.dxt, m, n_ux, B.dxdf, B.dex, B.dspread);
    k_split_rows<<<(unsigned)((wg * 32 + 255) / 256), 256, 0, s>>>(B.dg, m, (int)R, B.dgdf, B.deg, B.dspread + 1);
    count_launch(2);
  }
  dim3 g1((unsigned)((R + S1_BN - 1) / S1_BN), (n_ux + S1_BM - 1) / S1_BM);
  dim3 gdf((unsigned)((R + DF_BN - 1) / DF_BN), (n_ux + DF_BM - 1) / DF_BM);
  {
    ProfScope ps(PF_FF_CONTRACT, s, 16.0 * ((double)n_ux * m + (double)R * m + (double)n_ux * R),
                 8.0 * (double)n_ux * (double)R * m);
    // exactly one of the two writes T (device-side range check on the spreads)
    k_ff_stage1_df<<<gdf, 256, 0, s>>>(B.dxdf, B.dex, n_ux, B.dgdf, B.deg, (int)R, nbk, B.dspread, B.dT);
    k_ff_stage1<<<g1, 256, 0, s>>>(B.dxt, n_ux, B.dg, (int)R, m, B.dT, B.dspread);
  }
  count_launch(2);
  const double hd = std::pow(L.h, d);
  const double k2 = P->prob.k * P->prob.k;
  double2 pref = make_double2(k2 * hd * std::cos(d * P->prob.gamma), k2 * hd * std::sin(d * P->prob.gamma));
  if (d == 2)
    k_ff_stage2<2><<<n_ang, 256, 0, s>>>(B.dT, B.dxr, B.ds1, B.dyt, B.dzt, m, pref, F, F_exp, F_exp != nullptr,
                                         B.dmisc + 1);
  else
    k_ff_stage2<3><<<n_ang, 256, 0, s>>>(B.dT, B.dxr, B.ds1, B.dyt, B.dzt, m, pref, F, F_exp, F_exp != nullptr,
                                         B.dmisc + 1);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "far field kernels");
  if (scaled) {
    int flag = 0;
    if ((e = cudaMemcpyAsync(&flag, B.dmisc + 1, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "far field flag");
    *scaled = flag != 0;
  }
  return CSFF_OK;
}

}  // namespace csff
