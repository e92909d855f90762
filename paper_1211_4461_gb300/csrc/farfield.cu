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
#include <cuda_bf16.h>

#include <cmath>
#include <map>
#include <vector>

#include "csff_internal.h"
#include "df_bits.cuh"

namespace csff {
namespace {

// frexp's exponent of max(|re|, |im|), plus one, from the IEEE fields: -3999 for
// zero; a non-finite component counts as exponent 0
__device__ __forceinline__ int cexp2(double2 v) {
  const bool nzx = ((unsigned long long)__double_as_longlong(v.x) & bits::ABS_MASK) != 0;
  const bool nzy = ((unsigned long long)__double_as_longlong(v.y) & bits::ABS_MASK) != 0;
  int e = -4000;
  if (nzx) e = max(e, bits::exp_field(v.x) == 0x7ff ? 0 : bits::frexp_exp(v.x));
  if (nzy) e = max(e, bits::exp_field(v.y) == 0x7ff ? 0 : bits::frexp_exp(v.y));
  return e + 1;
}

// g = chi (u_in + u) at every interior node, and the largest frexp exponent of
// max(|Re g|, |Im g|) over the field (atomicMax into *emax, which the caller
// sets to -2000; 4000 when a component is not finite, -2000 for zero).
struct Tabs8 { const double2* p[8]; };

__global__ void k_fill_int(int* p, int v) { *p = v; }

__device__ __forceinline__ int value_exp(double2 x) {
  const int Ex = bits::exp_field(x.x), Ey = bits::exp_field(x.y);
  if (Ex == 0x7ff || Ey == 0x7ff) return 4000;
  const bool nzx = ((unsigned long long)__double_as_longlong(x.x) & bits::ABS_MASK) != 0;
  const bool nzy = ((unsigned long long)__double_as_longlong(x.y) & bits::ABS_MASK) != 0;
  return max(nzx ? bits::frexp_exp(x.x) : -2000, nzy ? bits::frexp_exp(x.y) : -2000);
}

template <int D>
__global__ void k_gfield(Tabs8 tabs, int n_gauss, const double2* __restrict__ uinc,
                         const double2* __restrict__ u, int m, double2* __restrict__ g, int* __restrict__ emax) {
  // g = chi u_in + chi u; chi u_in with each axis' Gaussian factor paired with
  // its incident-wave factor first (no partial product beyond the FP64 range).
  // The per-axis factors and pairs of the block's 32 columns are read and
  // formed once per block, those of its 8 rows (times the plane's, in 3D)
  // likewise, so a node costs two complex products per Gaussian.
  __shared__ double2 ex[8][32], eyz[8][8], px[8][32], pyz[8][8];
  __shared__ int wmax[8];
  const int t = threadIdx.y * 32 + threadIdx.x;
  for (int i = t; i < n_gauss * 40; i += 256) {
    const int q = i / 40, r = i % 40;
    const double2* E = tabs.p[q];
    if (r < 32) {
      const int x = blockIdx.x * 32 + r;
      const double2 f = x < m ? E[x] : make_double2(0, 0);
      ex[q][r] = f;
      px[q][r] = x < m ? cmul(f, uinc[x]) : make_double2(0, 0);
    } else {
      const int y = blockIdx.y * 8 + (r - 32);
      double2 f = y < m ? E[m + y] : make_double2(0, 0);
      double2 pf = y < m ? cmul(f, uinc[m + y]) : make_double2(0, 0);
      if (D == 3) {
        const double2 fz = E[2 * m + blockIdx.z];
        f = cmul(f, fz);
        pf = cmul(pf, cmul(fz, uinc[2 * m + blockIdx.z]));
      }
      eyz[q][r - 32] = f;
      pyz[q][r - 32] = pf;
    }
  }
  __syncthreads();
  const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y;
  const int iz = (D == 3) ? (int)blockIdx.z : 0;
  int e = -2000;
  if (ix < m && iy < m) {
    const long long idx = ((long long)iz * m + iy) * m + ix;
    double2 chi = make_double2(0, 0), cu = make_double2(0, 0);
    for (int q = 0; q < n_gauss; ++q) {
      chi = cadd(chi, cmul(ex[q][threadIdx.x], eyz[q][threadIdx.y]));
      cu = cadd(cu, cmul(px[q][threadIdx.x], pyz[q][threadIdx.y]));
    }
    const double2 v = cadd(cu, cmul(chi, u[idx]));
    g[idx] = v;
    e = value_exp(v);
  }
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (threadIdx.x == 0) wmax[threadIdx.y] = e;
  __syncthreads();
  if (t == 0) {
    int b = wmax[0];
    for (int w = 1; w < 8; ++w) b = max(b, wmax[w]);
    atomicMax(emax, b);
  }
}

// Phase tables P(a, x_i) = exp(-i k e^{i gamma} a x_i) = exp(k a x_i (sin g - i cos g)):
// one CTA per row (a distinct alpha_x; or an angle, whose y (and z) rows it
// fills).  The exponentials are evaluated exactly only at every PT_B-th node
// and for the PT_B offsets r h; each entry is then one complex product
// P(x_{jB + r}) = P(x_{jB}) P(r h), with two roundings more than a direct
// evaluation and a sixteenth of its FP64 transcendentals.  x rows carry the
// stage-1 range scale 2^-s1 (chosen from the a-priori bound on |T|).
constexpr int PT_B = 32;
size_t phase_tables_smem(int m) { return sizeof(double2) * 2 * ((m + PT_B - 1) / PT_B + PT_B); }

__global__ void __launch_bounds__(256) k_phase_tables(const double* __restrict__ ux, int n_ux,
                                                      const double* __restrict__ alpha, int n_ang, int dim, int m,
                                                      double lo, double h, double k, double sg, double cg,
                                                      const int* __restrict__ gmax, double2* __restrict__ xtab,
                                                      double2* __restrict__ ytab, double2* __restrict__ ztab,
                                                      int* __restrict__ s1, int* __restrict__ flag) {
  extern __shared__ double2 ptab[];        // per table: nb block values, then PT_B offset values
  const int row = blockIdx.x;
  const int nb = (m + PT_B - 1) / PT_B, W = nb + PT_B;
  const double LN2 = 0.69314718055994530942;
  int ntab, s = 0;
  double av[2] = {0.0, 0.0};
  double2* out[2] = {nullptr, nullptr};
  if (row < n_ux) {
    ntab = 1;
    av[0] = ux[row];
    out[0] = xtab + (long long)row * m;
    const double xmax = fmax(av[0] * (lo + h), av[0] * (lo + (double)m * h));   // max_i a x_i
    const int bx = (int)ceil(k * sg * xmax / LN2) + 1;
    int lm = 0;
    while ((1 << lm) < m) ++lm;
    s = bx + *gmax + lm + 2 - 1020;
    s = s > 0 ? s : 0;
    if (threadIdx.x == 0) {
      s1[row] = s;
      if (s > 0) atomicOr(flag, 1);
    }
  } else {
    const int ar = row - n_ux;
    if (ar >= n_ang) return;
    ntab = dim - 1;
    for (int c = 1; c < dim; ++c) av[c - 1] = alpha[(long long)ar * dim + c];
    out[0] = ytab + (long long)ar * m;
    out[1] = ztab + (long long)ar * m;
  }
  for (int q = threadIdx.x; q < ntab * W; q += blockDim.x) {
    const int tb = q / W, j = q - tb * W;
    const double a = av[tb];
    double x, sub = 0.0;
    if (j < nb) {
      x = lo + (double)(j * PT_B + 1) * h;
      sub = (double)s * LN2;
    } else {
      x = (double)(j - nb) * h;
    }
    const double mag = exp(k * sg * a * x - sub);
    double sn, cs;
    sincos(k * cg * a * x, &sn, &cs);
    ptab[q] = make_double2(mag * cs, -mag * sn);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < ntab * m; q += blockDim.x) {
    const int tb = q / m, i = q - tb * m;
    out[tb][i] = cmul(ptab[tb * W + i / PT_B], ptab[tb * W + nb + i % PT_B]);
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
// (x, y) summed over the block in the order bred uses, the result in thread
// 0 only: one pass for both components and no FP64 work for the other threads
__device__ __forceinline__ double2 bsum2_to0(double x, double y, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_double2(x, y);
  __syncthreads();
  double2 v = make_double2(0.0, 0.0);
  if (threadIdx.x == 0) {
    v = sh[0];
    for (int j = 1; j < (int)(blockDim.x >> 5); ++j) {
      v.x = v.x + sh[j].x;
      v.y = v.y + sh[j].y;
    }
  }
  return v;
}
struct MaxI { __device__ int operator()(int a, int b) const { return a > b ? a : b; } };

// Stage 2: one block per angle.
template <int D>
__global__ void k_ff_stage2(const double2* __restrict__ T, const int* __restrict__ xrow,
                            const int* __restrict__ s1, const double2* __restrict__ ytab,
                            const double2* __restrict__ ztab, int m, double2 pref,
                            double2* __restrict__ F, int* __restrict__ Fexp, int write_exp,
                            int* __restrict__ flag) {
  __shared__ int shi[32];
  __shared__ double2 shd[32];
  const int a = blockIdx.x;
  const int kx = xrow[a];
  const long long R = (D == 3) ? (long long)m * m : m;
  const double2* Tr = T + (long long)kx * R;
  const double2* yr = ytab + (long long)a * m;
  const double2* zr = ztab + (long long)a * m;
  int emax = -4000;
  // R = m (2D) or m^2 (3D) stays well inside int
  for (int r = threadIdx.x; r < (int)R; r += blockDim.x) {
    const int iy = (D == 3) ? r % m : r, iz = (D == 3) ? r / m : 0;
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
  for (int r = threadIdx.x; r < (int)R; r += blockDim.x) {
    const int iy = (D == 3) ? r % m : r, iz = (D == 3) ? r / m : 0;
    double2 w = s2 > 0 ? cscale(yr[iy], sc) : yr[iy];    // the scale is 1 unless the sum could overflow
    if (D == 3) w = cmul(w, zr[iz]);
    double2 t = Tr[r];
    ax = fma(w.x, t.x, fma(-w.y, t.y, ax));
    ay = fma(w.x, t.y, fma(w.y, t.x, ay));
  }
  const double2 axy = bsum2_to0(ax, ay, shd);
  if (threadIdx.x == 0) {
    double2 f = cmul(pref, axy);
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

// s += a * b in double-float for two sums at once (lane j of every pair holds
// sum j; one packed two-lane FP32 instruction per step, rounded per lane):
// the leading product p = a.hi b.hi and its exact error by FMA plus the cross
// terms a.hi b.lo + a.lo b.hi; s.hi + p by TwoSum (Knuth), whose error and the
// product's error collect in s.lo (s kept unnormalised).
__device__ __forceinline__ void df_mac2(float2& sh, float2& sl, float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, __fmul2_rn(p, m1));     // exact error of the leading product
  e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
  const float2 t = __fadd2_rn(sh, p);                   // TwoSum(s.hi, p)
  const float2 v = __ffma2_rn(sh, m1, t);               // t - s.hi
  const float2 err = __fadd2_rn(__ffma2_rn(__ffma2_rn(v, m1, t), m1, sh), __ffma2_rn(v, m1, p));
  sh = t;
  sl = __fadd2_rn(sl, __fadd2_rn(err, e));
}

// one warp per (row, block): block exponent of |v| (upper bound), scaled
// double-float split, and the row-block spread (max - min exponent) into *spread.
// elo (block bounds for skipping negligible blocks, see k_ff_df_skip):
// lo_min != 0 writes the smallest exponent of the block's entries inside the
// grid (-100000 if one is zero: max(|re|, |im|) >= 2^(e-1) for every entry),
// else the largest (-100000 for an all-zero block: some entry reaches 2^(e-1)).
__global__ void k_split_rows(const double2* __restrict__ v, int m, int nrows, float4* __restrict__ vdf,
                             float2* __restrict__ vsum, int* __restrict__ ev, int* __restrict__ spread,
                             int* __restrict__ elo, int lo_min) {
  // the spread is reduced over the CTA before one atomic (a per-warp atomic on
  // the one counter serialises in L2)
  __shared__ int wsp[8];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nb = (m + DKB - 1) / DKB;
  if (threadIdx.x < 8) wsp[threadIdx.x] = 0;
  __syncthreads();
  const bool active = warp < nrows * nb;        // warp-uniform
  const int row = active ? warp / nb : 0, b = active ? warp % nb : 0;
  const int i = b * DKB + lane;
  double2 x = (active && i < m) ? v[(long long)row * m + i] : make_double2(0, 0);
  // exponent of max(|re|, |im|) from the IEEE fields: the larger of the two
  // components' frexp exponents (a non-finite component marks the row bad)
  const bool fin = bits::exp_field(x.x) != 0x7ff && bits::exp_field(x.y) != 0x7ff;
  const bool nzx = ((unsigned long long)__double_as_longlong(x.x) & bits::ABS_MASK) != 0;
  const bool nzy = ((unsigned long long)__double_as_longlong(x.y) & bits::ABS_MASK) != 0;
  const bool pos = fin && (nzx || nzy);
  int e = pos ? max(nzx ? bits::frexp_exp(x.x) : -100000, nzy ? bits::frexp_exp(x.y) : -100000) : -100000;
  int emin = pos ? e : 100000;
  int elow = (i < m) ? e : 100000;               // -100000 for a zero entry; padding lanes ignored
  for (int o = 16; o > 0; o >>= 1) {
    e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    elow = min(elow, __shfl_xor_sync(0xffffffffu, elow, o));
  }
  const bool bad = __any_sync(0xffffffffu, !fin);   // non-finite: the FP64 kernel runs
  const int eb = (e == -100000 || bad) ? 0 : e;
  if (active && lane == 0) {
    ev[(long long)row * nb + b] = eb;
    if (elo) elo[(long long)row * nb + b] = lo_min ? elow : e;
    wsp[threadIdx.x >> 5] = bad ? DF_NONFINITE : ((e == -100000) ? 0 : e - emin);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int sp = 0;
    for (int w = 0; w < 8; ++w) sp = max(sp, wsp[w]);
    if (sp > 0) atomicMax(spread, sp);
  }
  // the scaled splits of re, im and re + im (Gauss's three-product complex
  // multiply); the scale applies to the values themselves, since 2^-eb alone
  // overflows for subnormal blocks
  const bool zero = e == -100000 || bad;
  float2 re = make_float2(0.f, 0.f), im = re, sm = re;
  if (!zero) {
    re = bits::split_scaled(x.x, eb);
    im = bits::split_scaled(x.y, eb);
    sm = eb <= 1000 ? bits::split_scaled(x.x + x.y, eb)      // RN(x + y) 2^-eb = RN(x 2^-eb + y 2^-eb)
                    : bits::split_scaled(ldexp(x.x, -eb) + ldexp(x.y, -eb), 0);
  }
  if (active) {
    const long long o = (long long)row * nb * DKB + b * DKB + lane;
    vdf[o] = make_float4(re.x, re.y, im.x, im.y);
    vsum[o] = sm;
  }
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

__device__ __forceinline__ void dfacc_merge3(dfacc& a1, dfacc& a2, dfacc& a3, df s1, df s2, df s3, int Es) {
  if (s1.hi == 0.f && s2.hi == 0.f && s3.hi == 0.f && s1.lo == 0.f && s2.lo == 0.f && s3.lo == 0.f) return;
  const int En = max(a1.E, Es);                    // the three share one exponent
  const float fa = pow2f_neg(a1.E - En), fs = pow2f_neg(Es - En);
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
  add(a1, s1);
  add(a2, s2);
  add(a3, s3);
}

// T[k][rho] over blocks; 16 (k) x 32 (rho) output tile per CTA of 128 threads,
// 2 x 2 outputs per thread (each operand value loaded from shared memory
// serves two outputs); the 736 CTAs of the 1025^2 maps fit one wave at 5 per SM.
constexpr int DF_BM = 16, DF_BN = 32, DF_NT = 128;

// Complex products by Gauss's three multiplications: with p1 = ar br,
// p2 = ai bi, p3 = (ar + ai)(br + bi) summed separately, Re = S1 - S2 and
// Im = S3 - S1 - S2 (formed in FP64 at the end).  Three double-float
// multiply-adds per complex term instead of four; the rounding of each sum
// stays relative to the sum of its terms' magnitudes, all bounded by
// (|ar| + |ai|)(|br| + |bi|), so the error is still double-float-small
// against the sum of the terms' magnitudes.
// Negligible blocks of the contraction.  For an output T[k][rho] the sum of
// its terms' magnitudes is at least
//   2^L,  L = max_b (xlo[k][b] + ghi[rho][b] - 2)
// (xlo: smallest exponent of X's entries in block b, ghi: largest of g's), and
// block b adds at most 32 * 2 * 2^(ex[k][b] + eg[rho][b]) (ex, eg: the block
// exponents the split scales by).  A block whose bound lies 60 binades under
// L for every (k, rho) of a contraction tile is skipped by that tile: per
// angle the skipped terms of the far field stay below 2^-55 of the sum of the
// magnitudes of all its terms (the factor Y[alpha][rho] of stage 2 is common
// to both sides), far below the double-float rounding.  All-zero g blocks add
// nothing and set no constraint.  One CTA per tile of k_ff_stage1_df.
constexpr int DF_SKIP_MARGIN = 60;
constexpr int DF_SKIP_NB_SMEM = 96;      // block counts up to this stage the exponents in shared memory
// staged rows are (nb | 1) ints apart: lanes reading one column of 32 different
// rows then hit 32 different banks
__host__ __device__ constexpr size_t df_skip_smem(int nb) {
  return (size_t)(2 * DF_BM + 2 * DF_BN) * (nb <= DF_SKIP_NB_SMEM ? (nb | 1) : 0) * sizeof(int);
}
__global__ void k_ff_df_skip(const int* __restrict__ ex, const int* __restrict__ xlo, int M,
                             const int* __restrict__ eg, const int* __restrict__ ghi, int N, int nb,
                             unsigned char* __restrict__ skip) {
  __shared__ int Ls[DF_BM * DF_BN];
  extern __shared__ int sexp[];          // the tile's rows of ex, xlo, eg, ghi when nb is small
  const int m0 = blockIdx.y * DF_BM, n0 = blockIdx.x * DF_BN;
  constexpr int OUTSIDE = -(1 << 30);    // pair outside the output range: no constraint
  constexpr int UNKNOWN = -(1 << 29);    // no lower bound for the pair: nothing may be skipped
  const bool staged = nb <= DF_SKIP_NB_SMEM;
  const int ps = staged ? (nb | 1) : nb;   // row pitch of sx, sxl, sg, sgh
  const int* sx = ex + (long long)m0 * nb;
  const int* sxl = xlo + (long long)m0 * nb;
  const int* sg = eg + (long long)n0 * nb;
  const int* sgh = ghi + (long long)n0 * nb;
  if (staged) {
    int* t = sexp;
    for (int i = threadIdx.x; i < DF_BM * nb; i += blockDim.x) {
      const int row = i / nb, j = row * ps + i % nb;
      const bool in = m0 + row < M;
      t[j] = in ? sx[i] : 0;
      t[DF_BM * ps + j] = in ? sxl[i] : -100000;
    }
    for (int i = threadIdx.x; i < DF_BN * nb; i += blockDim.x) {
      const int row = i / nb, j = row * ps + i % nb;
      const bool in = n0 + row < N;
      t[2 * DF_BM * ps + j] = in ? sg[i] : 0;
      t[2 * DF_BM * ps + DF_BN * ps + j] = in ? sgh[i] : -100000;
    }
    __syncthreads();
    sx = t;
    sxl = t + DF_BM * ps;
    sg = t + 2 * DF_BM * ps;
    sgh = t + 2 * DF_BM * ps + DF_BN * ps;
  }
  for (int p = threadIdx.x; p < DF_BM * DF_BN; p += blockDim.x) {
    const int k = p / DF_BN, r = p % DF_BN;
    int L = OUTSIDE;
    if (m0 + k < M && n0 + r < N) {
      L = UNKNOWN;
      for (int b = 0; b < nb; ++b) {
        const int a = sxl[k * ps + b], g = sgh[r * ps + b];
        if (a > -100000 && g > -100000) L = max(L, a + g - 2);
      }
    }
    Ls[p] = L;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long long tile = (long long)blockIdx.y * gridDim.x + blockIdx.x;
  for (int b = warp; b < nb; b += nw) {
    int worst = OUTSIDE;                                // max over pairs of bound - L
    for (int p = lane; p < DF_BM * DF_BN; p += 32) {
      const int L = Ls[p];
      if (L == OUTSIDE) continue;
      const int k = p / DF_BN, r = p % DF_BN;
      if (sgh[r * ps + b] <= -100000) continue;        // zero block of g: adds nothing
      if (L == UNKNOWN) { worst = 1 << 20; continue; }
      worst = max(worst, sx[k * ps + b] + sg[r * ps + b] + 6 - L);
    }
    for (int o = 16; o > 0; o >>= 1) worst = max(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if (lane == 0) skip[tile * nb + b] = worst < -DF_SKIP_MARGIN ? 1 : 0;
  }
}

__global__ void __launch_bounds__(DF_NT, 5) k_ff_stage1_df(const float4* __restrict__ X, const float2* __restrict__ Xs,
                                                        const int* __restrict__ ex, int M,
                                                        const float4* __restrict__ G, const float2* __restrict__ Gs,
                                                        const int* __restrict__ eg, int N, int nb,
                                                        const int* __restrict__ spread,
                                                        const unsigned char* __restrict__ skip,
                                                        double2* __restrict__ T) {
  if (!df_selected(spread)) return;      // the FP64 kernel takes this launch
  __shared__ float4 As[DF_BM][DKB + 1];
  __shared__ float2 As2[DF_BM][DKB + 1];
  // g rows tx and tx + 16 side by side (the two outputs j of a thread), per
  // node: (re.hi, re.hi'), (re.lo, re.lo'), (im.hi, ..), (im.lo, ..), (sum.hi, ..), (sum.lo, ..)
  __shared__ float4 Bp[DF_BN / 2][DKB + 1][3];
  __shared__ int eA[DF_BM], eB[DF_BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;   // ty: 0..7, rows 2 ty and 2 ty + 1
  const int m0 = blockIdx.y * DF_BM, n0 = blockIdx.x * DF_BN;
  dfacc acc1[2][2], acc2[2][2], acc3[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      acc1[i][j] = dfacc{0.f, 0.f, -100000};
      acc2[i][j] = dfacc{0.f, 0.f, -100000};
      acc3[i][j] = dfacc{0.f, 0.f, -100000};
    }
  const unsigned char* tskip = skip + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * nb;
  for (int b = 0; b < nb; ++b) {
    if (tskip[b]) continue;              // negligible for every output of the tile (uniform)
    for (int i = tid; i < DF_BM * DKB; i += DF_NT) {
      int r = i / DKB, kk = i % DKB, gm = m0 + r;
      const long long o = ((long long)gm * nb + b) * DKB + kk;
      As[r][kk] = (gm < M) ? X[o] : make_float4(0, 0, 0, 0);
      As2[r][kk] = (gm < M) ? Xs[o] : make_float2(0, 0);
    }
    for (int i = tid; i < DF_BN * DKB; i += DF_NT) {
      int r = i / DKB, kk = i % DKB, gn = n0 + r;
      const long long o = ((long long)gn * nb + b) * DKB + kk;
      const float4 gv = (gn < N) ? G[o] : make_float4(0, 0, 0, 0);
      const float2 gs = (gn < N) ? Gs[o] : make_float2(0, 0);
      float* d = reinterpret_cast<float*>(&Bp[r & 15][kk][0]);
      const int ln = r >> 4;
      d[ln] = gv.x;
      d[2 + ln] = gv.y;
      d[4 + ln] = gv.z;
      d[6 + ln] = gv.w;
      d[8 + ln] = gs.x;
      d[10 + ln] = gs.y;
    }
    if (tid < DF_BM) eA[tid] = (m0 + tid < M) ? ex[(long long)(m0 + tid) * nb + b] : 0;
    if (tid >= 64 && tid < 64 + DF_BN) eB[tid - 64] = (n0 + tid - 64 < N) ? eg[(long long)(n0 + tid - 64) * nb + b] : 0;
    __syncthreads();
    // block sums of the thread's outputs (i, j): lane j of the pairs
    float2 h1[2], l1[2], h2[2], l2[2], h3[2], l3[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      h1[i] = l1[i] = h2[i] = l2[i] = h3[i] = l3[i] = make_float2(0.f, 0.f);
    }
#pragma unroll 4
    for (int kk = 0; kk < DKB; ++kk) {
      const float4 b0 = Bp[tx][kk][0], b1 = Bp[tx][kk][1], b2 = Bp[tx][kk][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float4 a = As[2 * ty + i][kk];
        const float2 a2 = As2[2 * ty + i][kk];
        df_mac2(h1[i], l1[i], make_float2(a.x, a.x), make_float2(a.y, a.y), make_float2(b0.x, b0.y),
                make_float2(b0.z, b0.w));
        df_mac2(h2[i], l2[i], make_float2(a.z, a.z), make_float2(a.w, a.w), make_float2(b1.x, b1.y),
                make_float2(b1.z, b1.w));
        df_mac2(h3[i], l3[i], make_float2(a2.x, a2.x), make_float2(a2.y, a2.y), make_float2(b2.x, b2.y),
                make_float2(b2.z, b2.w));
      }
    }
    df s1[2][2], s2[2][2], s3[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      s1[i][0] = df{h1[i].x, l1[i].x};
      s1[i][1] = df{h1[i].y, l1[i].y};
      s2[i][0] = df{h2[i].x, l2[i].x};
      s2[i][1] = df{h2[i].y, l2[i].y};
      s3[i][0] = df{h3[i].x, l3[i].x};
      s3[i][1] = df{h3[i].y, l3[i].y};
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
        dfacc_merge3(acc1[i][j], acc2[i][j], acc3[i][j], s1[i][j], s2[i][j], s3[i][j],
                     eA[2 * ty + i] + eB[tx + 16 * j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int gm = m0 + 2 * ty + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      const double S1 = (double)acc1[i][j].hi + (double)acc1[i][j].lo;
      const double S2 = (double)acc2[i][j].hi + (double)acc2[i][j].lo;
      const double S3 = (double)acc3[i][j].hi + (double)acc3[i][j].lo;
      T[(long long)gm * N + gn] = make_double2(ldexp(S1 - S2, acc1[i][j].E), ldexp(S3 - S1 - S2, acc1[i][j].E));
    }
  }
}

// ---- 3D stage A on the tensor cores ------------------------------------------
// T1[t][col] = sum_iz Pz[t][iz] g[iz][col] as a real GEMM D[col][j] = sum_k
// A[col][k] B[j][k] with k = 2 iz + (re, im):
//   A[col] = (g_re(iz), g_im(iz))_iz,  B[t]    = (P_re, -P_im)_iz  (Re T_t),
//                                      B[32+t] = (P_im,  P_re)_iz  (Im T_t).
// Each operand row is scaled by a power of two (per column of g, per z-row of
// P) and split into four BF16 terms v = v0 + v1 + v2 + v3 (32 significant
// bits, split4); the ten products with i + j <= 3 run as tcgen05.mma
// (kind::f16, BF16 inputs, FP32 accumulation in tensor memory), the (0,0)
// product in its own accumulator.  The accumulators are drained after every
// K chunk (32 z-nodes) into double-float sums in registers, so FP32
// accumulation never spans more than 64 K-values; the epilogue forms the
// sums in FP64 and applies the exponents.  Operands sit in shared memory in the
// 128-byte-swizzled K-major layout (8-row atoms of 1024 B, 16-byte chunk index
// XOR row mod 8): A is split and stored by the CTA's threads from g, B is
// pre-split and pre-swizzled in global memory.  Two pipeline stages; the MMAs
// of one stage run while the threads fill the other.
namespace tc {
constexpr int TM = 128;                       // GEMM rows (columns of g) per CTA
constexpr int TT = 32;                        // z-rows of P per launch (GEMM N = 2 TT = 64)
constexpr int KZ = 32;                        // z-nodes per K chunk (64 BF16 = one 128-byte row)
constexpr int NTHR = 256;
constexpr int A_SPLIT = TM * 128;             // bytes of one split of an A chunk
constexpr int B_SPLIT = 2 * TT * 128;         // bytes of one split of a B chunk
constexpr int NSPLIT = 4;                     // BF16 terms per operand value (32 significant bits)
constexpr int STAGE = NSPLIT * A_SPLIT + NSPLIT * B_SPLIT;
constexpr int SMEM = 2 * STAGE + 1024 + 64;
constexpr int SPREAD_LIMIT = 90;              // bits, see tc_selected
constexpr int NONFINITE = 100000;
constexpr long long WAIT_LIMIT = 1ll << 26;   // polls of an mbarrier before giving up
constexpr int ERR_TIMEOUT = 1;
}  // namespace tc

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled K-major tile
__device__ __forceinline__ int sw128(int r, int c) { return (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (leading offset unused for this layout), sm_100-family version
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// v (|v| < 1 after scaling) as three BF16 terms
__device__ __forceinline__ void split3(float v, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(v);
  const float r1 = __fsub_rn(v, __bfloat162float(a));
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(b)));
}

// e with |v| < 2^e from the biased exponent bits (v != 0; subnormals as -1022)
__device__ __forceinline__ int exp_bound(double v) {
  const int E = (__double2hiint(v) >> 20) & 0x7FF;
  return (E == 0 ? 1 : E) - 1022;
}

// float(v * 2^-e), round to nearest even, from the bit fields alone (no FP64
// arithmetic: this part runs FP64 at 1/61 of the FP32 rate).  Results below
// FP32's normal range become zero; v must be finite with |v| 2^-e < 2^127.
__device__ __forceinline__ float d2f_scaled(double v, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int hi = (unsigned int)(b >> 32);
  const int E = (int)((hi >> 20) & 0x7FF);
  const int Ef = E - e - 1023 + 127;
  if (E == 0 || Ef <= 0) return 0.f;
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  unsigned int f = ((unsigned int)Ef << 23) + (unsigned int)(mant >> 29);
  const unsigned int rem = (unsigned int)(mant & 0x1FFFFFFFull), halfway = 0x10000000u;
  f += (rem > halfway || (rem == halfway && (f & 1u))) ? 1u : 0u;   // a carry into the exponent is exact
  return __uint_as_float(f | (hi & 0x80000000u));
}

// v * 2^-e (|v| 2^-e < 1) as four BF16 terms with 32 significant bits: the
// top 24 bits of the FP64 significand, truncated (an FP32 value, split three
// ways exactly by split3), and the next bits rounded to one BF16 term.  The
// representation error is below 2^-32 |v 2^-e|.  Bit fields and FP32
// arithmetic only; values below FP32's normal range become zero.
__device__ __forceinline__ void split4(double v, int e, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c,
                                       __nv_bfloat16& d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const unsigned int hi32 = (unsigned int)(bits >> 32);
  const int E = (int)((hi32 >> 20) & 0x7FF);
  const int Ef = E - e - 1023 + 127;
  float head = 0.f, tail = 0.f;
  if (E != 0 && Ef > 0) {
    const unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
    const unsigned int sgn = hi32 & 0x80000000u;
    head = __uint_as_float(sgn | ((unsigned int)Ef << 23) | (unsigned int)(mant >> 29));
    // the 29 bits below the head: r 2^(Ef - 127 - 52), formed as
    // (r 2^-60) 2^(Ef - 119), both factors in FP32's normal range (Ef < 127)
    const unsigned int r = (unsigned int)(mant & 0x1FFFFFFFull);
    const float t = __fmul_rn(__fmul_rn((float)r, 0x1p-60f), __uint_as_float((unsigned int)(Ef - 119 + 127) << 23));
    tail = sgn ? -t : t;
  }
  split3(head, a, b, c);
  d = __float2bfloat16_rn(tail);
}

// 2^e as a double (e clamped to the normal range -1022..1023)
__device__ __forceinline__ double pow2d(int e) {
  e = max(-1022, min(e, 1023));
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// The tensor-core kernel runs when both operands are finite and the smaller
// of the two exponent spreads (max - min inside one scaled row) is at most
// SPREAD_LIMIT: every row then holds a product within 2^-(min spread + 2) of
// the row scales, so terms flushed below FP32's range cost at most 2^-126
// relative to it, far under the 2^-24 rounding of the split.
__device__ __forceinline__ bool tc_selected(const int* __restrict__ f) {
  return f[0] < tc::NONFINITE && f[1] < tc::NONFINITE && min(f[0], f[1]) <= tc::SPREAD_LIMIT;
}

// per column of g: exponent bound over z (of max(|re|, |im|) per node) and the
// spread -> flag[0]; a block covers 32 columns x 8 groups of z, reduced in
// shared memory
constexpr int GX_COLS = 32, GX_ZG = 8;
__global__ void __launch_bounds__(GX_COLS * GX_ZG) k_tc_gexp(const double2* __restrict__ g, int m, long long ncol,
                                                             int* __restrict__ ecol, int* __restrict__ flag) {
  __shared__ int smax[GX_ZG][GX_COLS], smin[GX_ZG][GX_COLS], sbad[GX_ZG][GX_COLS];
  const int cl = threadIdx.x % GX_COLS, zg = threadIdx.x / GX_COLS;
  const long long col = blockIdx.x * (long long)GX_COLS + cl;
  int emax = -100000, emin = 100000, bad = 0;
  if (col < ncol)
    for (int iz = zg; iz < m; iz += GX_ZG) {
      const double2 v = g[(long long)iz * ncol + col];
      const double a = fmax(fabs(v.x), fabs(v.y));
      bad |= !isfinite(a);
      if (a != 0.0) { const int e = exp_bound(a); emax = max(emax, e); emin = min(emin, e); }
    }
  smax[zg][cl] = emax;
  smin[zg][cl] = emin;
  sbad[zg][cl] = bad;
  __syncthreads();
  if (zg == 0) {
    for (int j = 1; j < GX_ZG; ++j) {
      emax = max(emax, smax[j][cl]);
      emin = min(emin, smin[j][cl]);
      bad |= sbad[j][cl];
    }
    int sp = 0;
    if (col < ncol) {
      ecol[col] = (emax == -100000) ? 0 : emax;
      sp = bad ? tc::NONFINITE : (emax == -100000 ? 0 : emax - emin);
    }
    for (int o = 16; o > 0; o >>= 1) sp = max(sp, __shfl_xor_sync(0xffffffffu, sp, o));
    if (cl == 0 && sp > 0) atomicMax(flag, sp);
  }
}

// per z-row of P: exponent bound and spread -> flag[1] (one warp per row)
__global__ void k_tc_pexp(const double2* __restrict__ zt, int T, int t0, int m, int* __restrict__ erow,
                          int* __restrict__ flag) {
  const int t = blockIdx.x, lane = threadIdx.x;
  int emax = -100000, emin = 100000;
  bool bad = false;
  if (t0 + t < T)
    for (int iz = lane; iz < m; iz += 32) {
      const double2 v = zt[(long long)(t0 + t) * m + iz];
      const double a = fmax(fabs(v.x), fabs(v.y));
      bad |= !isfinite(a);
      if (a != 0.0) { const int e = exp_bound(a); emax = max(emax, e); emin = min(emin, e); }
    }
  for (int o = 16; o > 0; o >>= 1) {
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    erow[t] = (emax == -100000) ? 0 : emax;
    atomicMax(flag + 1, bad ? tc::NONFINITE : (emax == -100000 ? 0 : emax - emin));
  }
}

// B operand: per K chunk c and split s, 64 rows x 128 B, pre-swizzled; one
// thread per (chunk, row, 16-byte chunk)
__global__ void k_tc_psplit(const double2* __restrict__ zt, int T, int t0, int m, int nkc,
                            const int* __restrict__ erow, unsigned char* __restrict__ Bg) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nkc * 2 * tc::TT * 8) return;
  const int q = id & 7, j = (id >> 3) % (2 * tc::TT), c = id / (2 * tc::TT * 8);
  const int t = j % tc::TT, im_row = j / tc::TT;
  __align__(16) __nv_bfloat16 v[tc::NSPLIT][8];
  const int er = erow[t];
  for (int e = 0; e < 8; ++e) {
    const int k = q * 8 + e, iz = c * tc::KZ + (k >> 1);
    double x = 0.0;
    if (t0 + t < T && iz < m) {
      const double2 p = zt[(long long)(t0 + t) * m + iz];
      // Re rows (P_re, -P_im), Im rows (P_im, P_re)
      x = im_row ? ((k & 1) ? p.x : p.y) : ((k & 1) ? -p.y : p.x);
    }
    split4(x, er, v[0][e], v[1][e], v[2][e], v[3][e]);
  }
  for (int sidx = 0; sidx < tc::NSPLIT; ++sidx) {
    unsigned char* dst = Bg + ((size_t)c * tc::NSPLIT + sidx) * tc::B_SPLIT + sw128(j, q);
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(v[sidx]);
  }
}

// (hi, lo) += x + y as double-float: x + y exactly by TwoSum, then TwoSum with
// hi; the errors collect in lo (non-contracting intrinsics keep each rounding)
__device__ __forceinline__ void df_accumulate(float& hi, float& lo, float x, float y) {
  const float s = __fadd_rn(x, y), bb = __fsub_rn(s, x);
  const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(y, bb));
  const float h = __fadd_rn(hi, s), b2 = __fsub_rn(h, hi);
  const float e2 = __fadd_rn(__fsub_rn(hi, __fsub_rn(h, b2)), __fsub_rn(s, b2));
  hi = h;
  lo = __fadd_rn(lo, __fadd_rn(e, e2));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < tc::WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(tc::NTHR, 1)
    k_ff3_stageA_tc(const double2* __restrict__ g, int m, long long ncol, int T, int t0, int nkc,
                    const unsigned char* __restrict__ Bg, const int* __restrict__ ecol,
                    const int* __restrict__ erow, int* __restrict__ flag, double2* __restrict__ T1) {
  if (!tc_selected(flag)) return;                  // the FP64 kernel takes this launch
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + 2 * tc::STAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(base + 2 * tc::STAGE + 32);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long col0 = (long long)blockIdx.x * tc::TM;
  const int rl = tid & (tc::TM - 1), half = tid >> 7;     // row of A and z half-chunk of this thread
  const long long col = col0 + rl;
  const bool colv = col < ncol;
  const int ecl = colv ? ecol[col] : 0;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  // instruction descriptor: FP32 accumulator, BF16 A and B, K-major, N = 64, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(2 * tc::TT >> 3) << 17) |
                         ((uint32_t)(tc::TM >> 4) << 24);
  // this thread's outputs: warp w holds rows 32 (w % 4) + lane (TMEM lanes) and
  // z-rows [16 (w / 4), +16); per output a double-float running sum of the
  // chunk sums (re, im)
  const int lg = warp & 3, th = warp >> 2;
  float acc_hi[2][16], acc_lo[2][16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc_hi[0][j] = acc_lo[0][j] = acc_hi[1][j] = acc_lo[1][j] = 0.f;
  bool ok = true;
  // Chunk c's ten products accumulate in FP32 in TMEM set c & 1 (columns
  // 128 (c & 1) + [0, 64): the (0,0) product, + [64, 128): the other nine),
  // starting from zero; while the tensor core works on chunk c, the threads
  // read chunk c - 1's two accumulators and add them into the double-float
  // sums.  FP32 accumulation thus spans 64 K-values (32 z-nodes) only.
  auto drain = [&](int cd) {
    const int sd = cd & 1;
    ok &= mbar_wait(smem_addr(&mbar[sd]), (uint32_t)((cd >> 1) & 1));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t ta = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(128 * sd);
    uint32_t r0[16], i0[16], r1[16], i1[16];
#define TC_LD16(dst, colo)                                                                                   \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
               : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]),          \
                 "=r"(dst[6]), "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]),          \
                 "=r"(dst[12]), "=r"(dst[13]), "=r"(dst[14]), "=r"(dst[15])                                     \
               : "r"(ta + (uint32_t)(colo)))
    TC_LD16(r0, 16 * th);
    TC_LD16(i0, tc::TT + 16 * th);
    TC_LD16(r1, 2 * tc::TT + 16 * th);
    TC_LD16(i1, 3 * tc::TT + 16 * th);
#undef TC_LD16
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      df_accumulate(acc_hi[0][j], acc_lo[0][j], __uint_as_float(r0[j]), __uint_as_float(r1[j]));
      df_accumulate(acc_hi[1][j], acc_lo[1][j], __uint_as_float(i0[j]), __uint_as_float(i1[j]));
    }
  };
  for (int c = 0; c < nkc; ++c) {
    const int st = c & 1;
    unsigned char* sA = base + st * tc::STAGE;
    unsigned char* sB = sA + tc::NSPLIT * tc::A_SPLIT;
    // stage st and TMEM set st were last used by chunk c - 2, whose MMAs the
    // drain of iteration c - 1 waited for
    // A: 16 z-nodes of this thread's column, 4 at a time -> one 16-byte chunk per split
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const int izl = half * 16 + qq * 4;
      __align__(16) __nv_bfloat16 v[tc::NSPLIT][8];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int iz = c * tc::KZ + izl + e;
        double2 x = make_double2(0.0, 0.0);
        if (colv && iz < m) x = g[(long long)iz * ncol + col];
        split4(x.x, ecl, v[0][2 * e], v[1][2 * e], v[2][2 * e], v[3][2 * e]);
        split4(x.y, ecl, v[0][2 * e + 1], v[1][2 * e + 1], v[2][2 * e + 1], v[3][2 * e + 1]);
      }
      const int off = sw128(rl, half * 4 + qq);
#pragma unroll
      for (int sidx = 0; sidx < tc::NSPLIT; ++sidx)
        *reinterpret_cast<uint4*>(sA + sidx * tc::A_SPLIT + off) = *reinterpret_cast<const uint4*>(v[sidx]);
    }
    // B: copy the pre-swizzled chunk
    {
      const uint4* src = reinterpret_cast<const uint4*>(Bg + (size_t)c * tc::NSPLIT * tc::B_SPLIT);
      uint4* dst = reinterpret_cast<uint4*>(sB);
      for (int i = tid; i < tc::NSPLIT * tc::B_SPLIT / 16; i += tc::NTHR) dst[i] = src[i];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the ten products of split terms i, j with i + j <= 3 (the rest are
      // below 2^-33 of each term)
      const int pa[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3}, pb[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
#pragma unroll
      for (int p = 0; p < 10; ++p) {
        const uint32_t dacc = tmem + (uint32_t)(128 * st) + (p == 0 ? 0u : (uint32_t)(2 * tc::TT));
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t ad = sw128_desc(smem_addr(sA + pa[p] * tc::A_SPLIT) + 32 * kk);
          const uint64_t bd = sw128_desc(smem_addr(sB + pb[p] * tc::B_SPLIT) + 32 * kk);
          const uint32_t acc = (kk > 0 || p > 1) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(dacc),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&mbar[st]))
                   : "memory");
    }
    __syncwarp();
    if (c >= 1) drain(c - 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  // the last chunk; its commit covers every MMA issued before it
  drain(nkc - 1);
  if (!ok) {
    atomicOr(flag + 2, tc::ERR_TIMEOUT);
    mbar_wait(smem_addr(&mbar[(nkc - 1) & 1]), (uint32_t)(((nkc - 1) >> 1) & 1));
  }
  if (ok) {
    const long long ocol = col0 + 32 * lg + lane;
    if (ocol < ncol) {
      const int ec = ecol[ocol];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int t = 16 * th + j;
        if (t0 + t >= T) continue;
        const int e = ec + erow[t];
        const double re = (double)acc_hi[0][j] + (double)acc_lo[0][j];
        const double im = (double)acc_hi[1][j] + (double)acc_lo[1][j];
        T1[(long long)(t0 + t) * ncol + ocol] =
            (e >= -1022 && e <= 1023) ? make_double2(re * pow2d(e), im * pow2d(e)) : make_double2(ldexp(re, e), ldexp(im, e));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// ---- 3D sum-factorised contraction --------------------------------------------
// stage A: T1[t][col] = sum_iz Pz[t][iz] g[iz][col] for a group of TB distinct
// z-components t (col = iy m + ix); each thread keeps TB sums in registers so
// g is streamed once per group.
template <int TB>
__global__ void __launch_bounds__(256) k_ff3_stageA(const double2* __restrict__ zt, int T, int t0,
                                                    const double2* __restrict__ g, int m, long long ncol,
                                                    double2* __restrict__ T1, const int* __restrict__ skip_if_tc) {
  if (skip_if_tc && tc_selected(skip_if_tc)) return;   // the tensor-core kernel wrote T1
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

// fraction of the double-float contraction's (tile, block) pairs that the last
// 2D far field computed (1 when the FP64 kernel ran or nothing was skipped)
csff_status far_field_executed(csff_plan* P, double* executed) {
  FFBuffers& B = P->ff;
  *executed = 1.0;
  if (!B.dskip || !B.dspread || B.skip_used == 0) return CSFF_OK;
  std::vector<unsigned char> h(B.skip_used);
  int sp[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(h.data(), B.dskip, h.size(), cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sp, B.dspread, sizeof(sp), cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_fail(e, "far-field work");
  const bool df = sp[0] < DF_NONFINITE && sp[1] < DF_NONFINITE && std::min(sp[0], sp[1]) <= DF_SPREAD_LIMIT;
  if (!df) return CSFF_OK;
  size_t run = 0;
  for (unsigned char c : h) run += c == 0;
  *executed = (double)run / (double)h.size();
  return CSFF_OK;
}

void free_ff_buffers(csff_plan* P) {
  FFBuffers& b = P->ff;
  for (void* p : {(void*)b.dg, (void*)b.dxt, (void*)b.dyt, (void*)b.dzt, (void*)b.dT, (void*)b.dal,
                  (void*)b.dux, (void*)b.dxr, (void*)b.ds1, (void*)b.dmisc, (void*)b.dxdf, (void*)b.dgdf, (void*)b.dxsm, (void*)b.dgsm,
                  (void*)b.dex, (void*)b.deg, (void*)b.dspread, (void*)b.dtcb, (void*)b.dtce, (void*)b.dtcflag,
                  (void*)b.dxlo, (void*)b.dghi, (void*)b.dskip})
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
  k_fill_int<<<1, 1, 0, s>>>(B.dmisc, -2000);
  count_launch();
  if (d == 2) k_gfield<2><<<gg, gb, 0, s>>>(t, P->prob.n_gauss, P->uinc_tab, u, m, B.dg, B.dmisc);
  else k_gfield<3><<<gg, gb, 0, s>>>(t, P->prob.n_gauss, P->uinc_tab, u, m, B.dg, B.dmisc);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "g field");
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
      const bool use_tc = P->ff_mode == CSFF_FF_TC_BF16X4;
      const int nkc = (m + tc::KZ - 1) / tc::KZ;
      if (use_tc) {
        if ((e = ensure((void**)&B.dtcb, B.tcb, (size_t)nkc * tc::NSPLIT * tc::B_SPLIT, P)) != cudaSuccess ||
            (e = ensure((void**)&B.dtce, B.tce, sizeof(int) * ((size_t)ncol + tc::TT), P)) != cudaSuccess)
          return cuda_fail(e, "far field scratch");
        if (!B.dtcflag && (e = cudaMalloc((void**)&B.dtcflag, 3 * sizeof(int))) != cudaSuccess)
          return cuda_fail(e, "far field scratch");
        if ((e = cudaFuncSetAttribute(k_ff3_stageA_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM)) !=
                cudaSuccess ||
            (e = cudaMemsetAsync(B.dtcflag, 0, 3 * sizeof(int), s)) != cudaSuccess)
          return cuda_fail(e, "far field tensor-core set-up");
        k_tc_gexp<<<(unsigned)((ncol + GX_COLS - 1) / GX_COLS), GX_COLS * GX_ZG, 0, s>>>(B.dg, m, ncol, B.dtce,
                                                                                         B.dtcflag);
        count_launch();
      }
      {
        ProfScope ps(PF_FF_CONTRACT, s, 16.0 * ((double)n_uz * m + (double)ncol * m + (double)n_uz * ncol),
                     8.0 * (double)n_uz * (double)ncol * m);
        if (use_tc) {
          // per group of 32 z-rows: exponents and split phases, the tensor-core
          // kernel, and the FP64 kernel, which returns at once unless the range
          // check turned the tensor-core kernel away
          for (int t0 = 0; t0 < n_uz; t0 += tc::TT) {
            int* erow = B.dtce + ncol;
            if ((e = cudaMemsetAsync(B.dtcflag + 1, 0, sizeof(int), s)) != cudaSuccess)
              return cuda_fail(e, "memset");
            k_tc_pexp<<<tc::TT, 32, 0, s>>>(B.dxt, n_uz, t0, m, erow, B.dtcflag);
            const int nth = nkc * 2 * tc::TT * 8;
            k_tc_psplit<<<(nth + 255) / 256, 256, 0, s>>>(B.dxt, n_uz, t0, m, nkc, erow, B.dtcb);
            k_ff3_stageA_tc<<<(unsigned)((ncol + tc::TM - 1) / tc::TM), tc::NTHR, tc::SMEM, s>>>(
                B.dg, m, ncol, n_uz, t0, nkc, B.dtcb, B.dtce, erow, B.dtcflag, T1);
            for (int tb = t0; tb < std::min(n_uz, t0 + tc::TT); tb += 16)
              k_ff3_stageA<16><<<(unsigned)((ncol + 255) / 256), 256, 0, s>>>(B.dxt, n_uz, tb, B.dg, m, ncol, T1,
                                                                              B.dtcflag);
            count_launch(3 + (std::min(n_uz, t0 + tc::TT) - t0 + 15) / 16);
          }
        } else {
          for (int t0 = 0; t0 < n_uz; t0 += 16)
            k_ff3_stageA<16><<<(unsigned)((ncol + 255) / 256), 256, 0, s>>>(B.dxt, n_uz, t0, B.dg, m, ncol, T1,
                                                                            nullptr);
          count_launch((n_uz + 15) / 16);
        }
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
      count_launch(3);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "far field 3D kernels");
      if (use_tc) {
        int fl[3] = {0, 0, 0};
        if ((e = cudaMemcpyAsync(fl, B.dtcflag, sizeof(fl), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
          return cuda_fail(e, "far field tensor-core status");
        if (fl[2] & tc::ERR_TIMEOUT) {
          set_error("tensor-core far field: an mbarrier wait ran out");
          return CSFF_ERR_TIMEOUT;
        }
      }
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
  k_phase_tables<<<n_ux + n_ang, 256, phase_tables_smem(m), s>>>(B.dux, n_ux, B.dal, n_ang, d, m, P->prob.box_lo,
                                                                 L.h, P->prob.k, sg, cg, B.dmisc, B.dxt, B.dyt,
                                                                 B.dzt, B.ds1, B.dmisc + 1);
  count_launch();
  // operands of the double-float contraction
  const int nbk = (m + DKB - 1) / DKB;
  if ((e = ensure((void**)&B.dxdf, B.xdf, sizeof(float4) * (size_t)n_ux * nbk * DKB, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dgdf, B.gdf, sizeof(float4) * (size_t)R * nbk * DKB, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dxsm, B.xsm, sizeof(float2) * (size_t)n_ux * nbk * DKB, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dgsm, B.gsm, sizeof(float2) * (size_t)R * nbk * DKB, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dex, B.exs, sizeof(int) * (size_t)n_ux * nbk, P)) != cudaSuccess ||
      (e = ensure((void**)&B.deg, B.egs, sizeof(int) * (size_t)R * nbk, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dxlo, B.xlo, sizeof(int) * (size_t)n_ux * nbk, P)) != cudaSuccess ||
      (e = ensure((void**)&B.dghi, B.ghi, sizeof(int) * (size_t)R * nbk, P)) != cudaSuccess)
    return cuda_fail(e, "far field scratch");
  if (!B.dspread && (e = cudaMalloc((void**)&B.dspread, 2 * sizeof(int))) != cudaSuccess)
    return cuda_fail(e, "far field scratch");
  if ((e = cudaMemsetAsync(B.dspread, 0, 2 * sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "memset");
  {
    const long long wx = (long long)n_ux * nbk, wg = (long long)R * nbk;
    k_split_rows<<<(unsigned)((wx * 32 + 255) / 256), 256, 0, s>>>(B.dxt, m, n_ux, B.dxdf, B.dxsm, B.dex,
                                                                   B.dspread, B.dxlo, 1);
    k_split_rows<<<(unsigned)((wg * 32 + 255) / 256), 256, 0, s>>>(B.dg, m, (int)R, B.dgdf, B.dgsm, B.deg,
                                                                   B.dspread + 1, B.dghi, 0);
    count_launch(2);
  }
  dim3 g1((unsigned)((R + S1_BN - 1) / S1_BN), (n_ux + S1_BM - 1) / S1_BM);
  dim3 gdf((unsigned)((R + DF_BN - 1) / DF_BN), (n_ux + DF_BM - 1) / DF_BM);
  if ((e = ensure((void**)&B.dskip, B.skip, (size_t)gdf.x * gdf.y * nbk, P)) != cudaSuccess)
    return cuda_fail(e, "far field scratch");
  k_ff_df_skip<<<gdf, 256, df_skip_smem(nbk), s>>>(B.dex, B.dxlo, n_ux, B.deg, B.dghi, (int)R, nbk, B.dskip);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "far-field skip flags");
  B.skip_used = (size_t)gdf.x * gdf.y * nbk;
  {
    ProfScope ps(PF_FF_CONTRACT, s, 16.0 * ((double)n_ux * m + (double)R * m + (double)n_ux * R),
                 8.0 * (double)n_ux * (double)R * m);
    // exactly one of the two writes T (device-side range check on the spreads)
    k_ff_stage1_df<<<gdf, DF_NT, 0, s>>>(B.dxdf, B.dxsm, B.dex, n_ux, B.dgdf, B.dgsm, B.deg, (int)R, nbk, B.dspread,
                                         B.dskip, B.dT);
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
