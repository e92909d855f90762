// Tile bodies of the fused 2D V(1,1) red-black Gauss-Seidel cycle (Sec. 4),
// shared by the per-level kernels (mg_fused.cu) and the persistent batched
// kernel (batch.cu).
//
//   down tile:   one RB-GS sweep on A_l u = b_l over a tile plus halo, the
//                residual on the tile, full weighting into b_{l+1}
//   up tile:     u += P e_{l+1}, one RB-GS sweep
//   coarse block: every level from lc to the coarsest in one CTA
//
// COH selects loads for data written by other CTAs earlier in the same launch
// (the persistent kernel): those go through L2 (ld.global.cg), never through
// the non-coherent read-only path.
#pragma once

#include "csff_internal.h"

namespace csff {
namespace tiles {

// Tile geometry for TC coarse points per tile side: the tile owns FT = 2 TC
// fine points per side; down window fine [2P0-3, 2P0+2TC+3], up window fine
// [2P0-2, 2P0+2TC+2], coarse window for up [P0-2, P0+TC+1].
template <int TC> struct Geo {
  static constexpr int FT = 2 * TC;
  static constexpr int DW = FT + 7;
  static constexpr int UW = FT + 5;
  static constexpr int EW = TC + 4;
};
constexpr int NT = 256;

// Coefficients of one fine level as the tile bodies see them: the diagonal
// d = 2D c - q and its inverse.  FP64 cycles read the plan's FP64 tables
// (q, dinv); FP32 cycles form them from separable per-axis factors,
//   q(z) = k^2 + sum_g X_g[ix] Y_g[iy],
//   X_g = 2^-s_g k^2 A_g e^{-(z_x - c_gx)^2 / w_g},  Y_g = 2^s_g e^{-(z_y - c_gy)^2 / w_g}
// (s_g balances the two factors' ranges), which leaves the RHS and the iterate
// as the only per-point streams of an FP32 tile.
template <typename T> struct LevelCoef {
  const cx<T>* q = nullptr;      // stored q (FP64 cycles)
  const cx<T>* dinv = nullptr;   // stored 1/d (FP64 cycles)
  const cx<T>* fac = nullptr;    // [ng][2][m] factors X_g, Y_g (FP32 cycles)
  int ng = 0;
  T k2 = 0;
};
template <typename T> constexpr bool formed_coef() { return sizeof(T) == 4; }

// Shared-memory windows are stored split by colour: window point (wx, wy)
// sits in plane (wx + wy) & 1, row wy, slot wx >> 1, with HS = (W + 1) / 2
// slots a row, rows P elements apart and planes PLANE apart.  A point in slot
// j of its row (wx = 2 j + o) finds its four neighbours in the other plane:
// slots j + o - 1 and j + o of the same row and slot j of the rows above and
// below, so a warp working along a row touches consecutive words.
//
// Row pitch of the FP32 down windows (ES = 8-byte elements): with P = HS the
// thread segments of a pass, which start an even number of rows apart, land
// on the same banks; a bank model of every pass of the tiles (each warp
// access costs as many wavefronts as the busiest bank pair has distinct
// words) gives 22-23 % fewer wavefronts with P = 21 for the 39-wide window
// and P = 14 with planes one element further apart for the 23-wide one.  The
// up windows gain nothing, and the FP64 windows stay unpadded, which keeps
// their CTAs per SM.
template <int W, int ES> struct RBPad {
  static constexpr int P = (ES == 8 && W == 39) ? 21 : (ES == 8 && W == 23) ? 14 : (W + 1) / 2;
  static constexpr int GAP = (ES == 8 && W == 23) ? 1 : 0;
};
template <int W, int ES = 8> struct RB {
  static constexpr int HS = (W + 1) / 2;
  static constexpr int P = RBPad<W, ES>::P;
  static constexpr int PLANE = W * P + RBPad<W, ES>::GAP;
  static constexpr int ELEMS = 2 * PLANE;
  // factor windows of one Gaussian: X_g split by the parity of wx (2 HS), Y_g (W)
  static constexpr int FACTOR = 2 * HS + W;
};
template <int W, int ES> __device__ __forceinline__ int rbi(int wx, int wy) {
  return ((wx + wy) & 1) * RB<W, ES>::PLANE + wy * RB<W, ES>::P + (wx >> 1);
}

template <int TC> __host__ __device__ constexpr int down_window(bool fp64) {
  return fp64 ? RB<Geo<TC>::DW, 16>::ELEMS : RB<Geo<TC>::DW, 8>::ELEMS;
}
template <int TC> __host__ __device__ constexpr int up_window(bool fp64) {
  return fp64 ? RB<Geo<TC>::UW, 16>::ELEMS : RB<Geo<TC>::UW, 8>::ELEMS;
}
// shared-memory elements (complex values) of one tile: iterate and RHS
// windows, then FP32 factor windows (ng Gaussians) or the FP64 1/d window
template <int TC> __host__ __device__ constexpr size_t down_smem_elems(int ng, bool fp64) {
  return (size_t)(fp64 ? 3 : 2) * down_window<TC>(fp64) + (fp64 ? 0 : (size_t)ng * RB<Geo<TC>::DW>::FACTOR);
}
template <int TC> __host__ __device__ constexpr size_t up_smem_elems(int ng, bool fp64) {
  return (size_t)(fp64 ? 3 : 2) * up_window<TC>(fp64) + Geo<TC>::EW * Geo<TC>::EW +
         (fp64 ? 0 : (size_t)ng * RB<Geo<TC>::UW>::FACTOR);
}

template <typename T>
__device__ __forceinline__ cx<T> zero_c() { return mk<cx<T>>((T)0, (T)0); }

// Complex arithmetic of the tiles with every rounding spelled out (round-to-
// nearest intrinsics are never contracted or reassociated by the compiler), so
// the per-level kernels and the persistent batched kernel, which inline the
// same tile bodies into different code, produce identical bits.
// The FP32 element-wise forms use the packed two-lane instructions (one
// instruction for both parts, the same rounding per part); a - b is
// fma(b, -1, a), exact product and one rounding.
__device__ __forceinline__ float2 xadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 xadd(double2 a, double2 b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 xsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 xsub(double2 a, double2 b) { return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)); }
__device__ __forceinline__ float2 xmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double2 xmul(double2 a, double2 b) {
  return make_double2(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 xscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ double2 xscale(double2 a, double s) { return make_double2(__dmul_rn(a.x, s), __dmul_rn(a.y, s)); }
// a + s b for a real s, one rounding per part
__device__ __forceinline__ float2 xfma_r(float2 a, float2 b, float s) { return __ffma2_rn(b, make_float2(s, s), a); }
__device__ __forceinline__ double2 xfma_r(double2 a, double2 b, double s) {
  return make_double2(__fma_rn(b.x, s, a.x), __fma_rn(b.y, s, a.y));
}
// a + b c and a - b c as chains of fused multiply-adds (one rounding each)
__device__ __forceinline__ float2 xfma(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(b.x, c.x, __fmaf_rn(-b.y, c.y, a.x)), __fmaf_rn(b.x, c.y, __fmaf_rn(b.y, c.x, a.y)));
}
__device__ __forceinline__ double2 xfma(double2 a, double2 b, double2 c) {
  return make_double2(__fma_rn(b.x, c.x, __fma_rn(-b.y, c.y, a.x)), __fma_rn(b.x, c.y, __fma_rn(b.y, c.x, a.y)));
}
__device__ __forceinline__ float2 xfms(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(-b.x, c.x, __fmaf_rn(b.y, c.y, a.x)), __fmaf_rn(-b.x, c.y, __fmaf_rn(-b.y, c.x, a.y)));
}
__device__ __forceinline__ double2 xfms(double2 a, double2 b, double2 c) {
  return make_double2(__fma_rn(-b.x, c.x, __fma_rn(b.y, c.y, a.x)), __fma_rn(-b.x, c.y, __fma_rn(-b.y, c.x, a.y)));
}

template <bool COH, typename C>
__device__ __forceinline__ C ld(const C* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// 1/d for the smoother: reciprocal of |d|^2 by the hardware approximation
// (__fdividef, about 2 ulp), enough for an inverse diagonal that only scales
// the correction
__device__ __forceinline__ float2 crecip(float2 d) {
  const float r = __fdividef(1.f, __fmaf_rn(d.x, d.x, __fmul_rn(d.y, d.y)));
  return make_float2(__fmul_rn(d.x, r), -__fmul_rn(d.y, r));
}

// Asynchronous global -> shared copies of BYTES (4, 8 or 16) to a 32-bit
// shared-window address (formed once per loop, then advanced by constants),
// unconditional or zero-filled when !valid (no bytes are read then).
// Per-level kernels only: data written by other CTAs of the same launch (the
// persistent kernel) is read through L2.
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_async_s(uint32_t dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(gsrc), "n"(BYTES) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_sz(uint32_t dst, const void* gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(gsrc), "n"(BYTES),
               "r"(valid ? BYTES : 0)
               : "memory");
}

// Window of W x W fine points with origin (ox, oy) in the colour-split layout.
//  - Iterate: the black points (window colour 1) only.  A red-black sweep
//    never reads a red point's own old value, and the red half sweep computes
//    every red value read afterwards, so red slots are only set to zero where
//    they lie outside the domain (Dirichlet neighbours of black edge points).
//  - RHS (FP64: and 1/d) on window [1, W-2]^2, the points the sweeps update.
//  - FP32: per Gaussian X_g at wx = 2 j + o in slot o HS + j, then Y_g along wy.
// Points outside the interior read as zero.  Per-level kernels copy
// asynchronously and, with WAIT, wait for their copies before returning;
// without it the caller waits (after issuing more copies of its own).
template <typename T, int W, bool COH, bool WAIT = true>
__device__ __forceinline__ void load_window(int ox, int oy, int m, const cx<T>* u_in, bool zero_u,
                                            const cx<T>* b, const LevelCoef<T>& K, cx<T>* U, cx<T>* B,
                                            cx<T>* X) {
  using L = RB<W, (int)sizeof(cx<T>)>;
  constexpr int HS = L::HS, P = L::P, PL = L::PLANE, WI = W - 2;
  const bool inner = ox >= 0 && oy >= 0 && ox + W <= m && oy + W <= m;
  if constexpr (!COH) {
    // Per-level kernels: each thread owns one window column of each array and
    // walks the window rows an even stride apart, so a row's colour plane and
    // slot stay fixed and the shared and global addresses advance by
    // constants; every copy of the thread is in flight at once (one round trip
    // per tile).  Points outside the interior read as zero.  Element offsets
    // are 32-bit: a 2D plan has at most 15 levels, so m <= 32767 and every
    // offset (m + W) m stays below 2^31.  A tile whose window lies inside the
    // domain copies without any per-element test.
    constexpr int E = (int)sizeof(cx<T>);
    const int t = threadIdx.x;
    {
      // black plane: wx = 2 jj + (~wy & 1)
      constexpr int RS = (NT / HS) & ~1, NK = (W + RS - 1) / RS;
      constexpr uint32_t DSTEP = RS * P * E;
      const int r0 = t / HS, jj = t - r0 * HS;
      const int wx = 2 * jj + ((r0 & 1) ^ 1);
      if (r0 < RS && wx < W) {
        const int fx = ox + wx, gstep = RS * m;
        const uint32_t dst = smem_addr(U + PL + r0 * P + jj);
        const int g = (oy + r0) * m + fx;
        if (inner && !zero_u) {
#pragma unroll
          for (int k = 0; k < NK; ++k)
            if (r0 + k * RS < W) cp_async_s<E>(dst + k * DSTEP, u_in + (g + k * gstep));
        } else {
          const bool xin = !zero_u && fx >= 0 && fx < m;
#pragma unroll
          for (int k = 0; k < NK; ++k) {
            const int wy = r0 + k * RS;
            if (wy < W) {
              const int fy = oy + wy;
              const bool in = xin && fy >= 0 && fy < m;
              cp_async_sz<E>(dst + k * DSTEP, u_in + (in ? g + k * gstep : 0), in);
            }
          }
        }
      }
    }
    if (!inner)
      for (int i = t; i < W * HS; i += NT) {                 // red plane: zero outside the domain
        const int wy = i / HS, j = i - wy * HS;
        const int fx = ox + 2 * j + (wy & 1), fy = oy + wy;
        if (!(fx >= 0 && fx < m && fy >= 0 && fy < m)) U[wy * P + j] = zero_c<T>();
      }
    {
      // right-hand side (FP64: and 1/d) on window [1, W-2]^2
      constexpr int RS = (NT / WI) & ~1, NK = (WI + RS - 1) / RS;
      constexpr uint32_t DSTEP = RS * P * E;
      const int r1 = t / WI, c1 = t - r1 * WI;
      if (r1 < RS) {
        const int wx = 1 + c1, wy0 = 1 + r1;
        const int fx = ox + wx, gstep = RS * m;
        const int d = rbi<W, E>(wx, wy0);
        const uint32_t dB = smem_addr(B + d), dX = smem_addr(X + d);
        const int g = (oy + wy0) * m + fx;
        if (inner) {
#pragma unroll
          for (int k = 0; k < NK; ++k)
            if (wy0 + k * RS <= WI) {
              cp_async_s<E>(dB + k * DSTEP, b + (g + k * gstep));
              if constexpr (!formed_coef<T>()) cp_async_s<E>(dX + k * DSTEP, K.dinv + (g + k * gstep));
            }
        } else {
          const bool xin = fx >= 0 && fx < m;
#pragma unroll
          for (int k = 0; k < NK; ++k) {
            const int wy = wy0 + k * RS;
            if (wy <= WI) {
              const int fy = oy + wy;
              const bool in = xin && fy >= 0 && fy < m;
              const int gk = in ? g + k * gstep : 0;
              cp_async_sz<E>(dB + k * DSTEP, b + gk, in);
              if constexpr (!formed_coef<T>()) cp_async_sz<E>(dX + k * DSTEP, K.dinv + gk, in);
            }
          }
        }
      }
    }
    if constexpr (formed_coef<T>()) {
      // factor windows: X_g at wx = 2 j + o in slot o HS + j, then Y_g along wy
      constexpr int FW = RB<W>::FACTOR;
      for (int i = t; i < K.ng * FW; i += NT) {
        const int gg = i / FW, r = i - gg * FW;
        int f;
        bool in;
        if (r < 2 * HS) {
          const int o = r >= HS ? 1 : 0;
          const int fx = ox + 2 * (r - o * HS) + o;
          in = fx >= 0 && fx < m;
          f = (gg * 2) * m + fx;
        } else {
          const int fy = oy + r - 2 * HS;
          in = fy >= 0 && fy < m;
          f = (gg * 2 + 1) * m + fy;
        }
        cp_async_sz<E>(smem_addr(X + i), K.fac + (in ? f : 0), in);
      }
    }
  } else {
    // The persistent kernel reads data other CTAs of the same launch wrote,
    // through L2 (ld.cg).  The same column-per-thread walk as above; each
    // thread issues all its loads into registers before it stores any, so a
    // window costs one round trip, not one per element.
    const int t = threadIdx.x;
    constexpr int RSU = (NT / HS) & ~1, NKU = (W + RSU - 1) / RSU;
    constexpr int RSB = (NT / WI) & ~1, NKB = (WI + RSB - 1) / RSB;
    constexpr int FW = RB<W>::FACTOR, NKF = formed_coef<T>() ? (8 * FW + NT - 1) / NT : 0;
    const int r0 = t / HS, jj = t - r0 * HS;
    const int wxu = 2 * jj + ((r0 & 1) ^ 1);
    const bool uact = r0 < RSU && wxu < W;
    const int r1 = t / WI, c1 = t - r1 * WI;
    const bool bact = r1 < RSB;
    cx<T> vu[NKU], vb[NKB], vx[NKB], vf[NKF > 0 ? NKF : 1];
    {
      const int fx = ox + wxu;
      const bool xin = uact && !zero_u && fx >= 0 && fx < m;
      const int g = (oy + r0) * m + fx;
#pragma unroll
      for (int k = 0; k < NKU; ++k) {
        const int wy = r0 + k * RSU, fy = oy + wy;
        const bool in = xin && wy < W && (inner || (fy >= 0 && fy < m));
        vu[k] = in ? ld<COH>(u_in + (g + k * RSU * m)) : zero_c<T>();
      }
    }
    {
      const int wx = 1 + c1, fx = ox + wx;
      const bool xin = bact && fx >= 0 && fx < m;
      const int g = (oy + 1 + r1) * m + fx;
#pragma unroll
      for (int k = 0; k < NKB; ++k) {
        const int wy = 1 + r1 + k * RSB, fy = oy + wy;
        const bool in = xin && wy <= WI && (inner || (fy >= 0 && fy < m));
        vb[k] = in ? ld<COH>(b + (g + k * RSB * m)) : zero_c<T>();
        if constexpr (!formed_coef<T>()) vx[k] = in ? ld<COH>(K.dinv + (g + k * RSB * m)) : zero_c<T>();
      }
    }
    if constexpr (formed_coef<T>()) {
      // factor windows (at most 8 Gaussians): X_g at wx = 2 j + o in slot
      // o HS + j, then Y_g along wy
#pragma unroll
      for (int k = 0; k < NKF; ++k) {
        const int i = t + k * NT;
        const int gg = i / FW, r = i - gg * FW;
        int f = 0;
        bool in = i < K.ng * FW;
        if (r < 2 * HS) {
          const int o = r >= HS ? 1 : 0;
          const int fx = ox + 2 * (r - o * HS) + o;
          in = in && fx >= 0 && fx < m;
          f = (gg * 2) * m + fx;
        } else {
          const int fy = oy + r - 2 * HS;
          in = in && fy >= 0 && fy < m;
          f = (gg * 2 + 1) * m + fy;
        }
        vf[k] = in ? ld<COH>(K.fac + f) : zero_c<T>();
      }
    }
    if (uact) {
#pragma unroll
      for (int k = 0; k < NKU; ++k)
        if (r0 + k * RSU < W) U[PL + (r0 + k * RSU) * P + jj] = vu[k];
    }
    if (bact) {
      const int d0 = rbi<W, (int)sizeof(cx<T>)>(1 + c1, 1 + r1);
#pragma unroll
      for (int k = 0; k < NKB; ++k)
        if (1 + r1 + k * RSB <= WI) {
          B[d0 + k * RSB * P] = vb[k];
          if constexpr (!formed_coef<T>()) X[d0 + k * RSB * P] = vx[k];
        }
    }
    if constexpr (formed_coef<T>()) {
#pragma unroll
      for (int k = 0; k < NKF; ++k)
        if (t + k * NT < K.ng * FW) X[t + k * NT] = vf[k];
    }
    if (!inner)
      for (int i = t; i < W * HS; i += NT) {               // red plane: zero outside the domain
        const int wy = i / HS, j = i - wy * HS;
        const int fx = ox + 2 * j + (wy & 1), fy = oy + wy;
        if (!(fx >= 0 && fx < m && fy >= 0 && fy < m)) U[wy * P + j] = zero_c<T>();
      }
  }
  if constexpr (!COH && WAIT) cp_async_wait_all();
}

// d = 4c - q = D0 - sum_g X_g Y_g (D0 = 4c - k^2) at the point in slot j
// (wx = 2 j + o) of window row wy, from the factor windows
template <int W>
__device__ __forceinline__ float2 formed_diag(const LevelCoef<float>& K, float2 D0, const float2* X, int o, int j,
                                              int wy) {
  constexpr int HS = RB<W>::HS, FW = RB<W>::FACTOR;
  float2 d = D0;
  for (int g = 0; g < K.ng; ++g) d = xfms(d, X[g * FW + o * HS + j], X[g * FW + 2 * HS + wy]);
  return d;
}

// Work split of a pass over R window rows: each thread takes slot column j of
// a segment of RS consecutive rows.  RS is even, so every segment starts on a
// row of LO's parity and the slot parity o of each row of the segment is a
// compile-time constant.
template <int W, int R> struct Seg {
  static constexpr int HS = RB<W>::HS;
  static constexpr int RS0 = (R + NT / HS - 1) / (NT / HS);
  static constexpr int RS = RS0 + (RS0 & 1);
  static constexpr int NSEG = (R + RS - 1) / RS;
  static_assert(NSEG * HS <= NT, "one segment per thread");
};

// One pass over the points of window colour COLOUR in window rows and columns
// [LO, HI] that lie inside the domain: a red-black Gauss-Seidel half sweep
//   u_j <- d_j^{-1} (b_j + c sum_nbr u),
// which equals u_j + d_j^{-1} (b_j - (A u)_j) for A u = d u - c sum_nbr u, or,
// with RESID, the residual r_j = b_j - (d_j u_j - c sum_nbr u) written over
// b_j.  The thread carries the other colour's slot-j values from row to row in
// registers (three loads and a store per point, all on consecutive words of a
// row).  Neighbour order of the sum: x-1, x+1, y-1, y+1.  G1: the level has a
// single Gaussian, whose x factors for the thread's two slot parities stay in
// registers.
template <typename T, int W, int COLOUR, int LO, int HI, bool RESID, bool G1>
__device__ __forceinline__ void rb_pass(int ox, int oy, int m, const LevelCoef<T>& K, cx<T> c, cx<T>* U,
                                        cx<T>* B, const cx<T>* X) {
  using C = cx<T>;
  using S = Seg<W, HI - LO + 1>;
  constexpr int HS = S::HS, RS = S::RS;
  constexpr int P = RB<W, (int)sizeof(C)>::P, PL = RB<W, (int)sizeof(C)>::PLANE;
  constexpr int OA = (COLOUR ^ LO) & 1;          // slot parity of the segment's even rows
  static_assert(LO >= 1 && HI <= W - 2, "neighbours inside the window");
  const int t = threadIdx.x;
  if (t >= S::NSEG * HS) return;
  const int seg = t / HS, j = t - seg * HS;
  const int y0 = LO + seg * RS;
  const int nrows = min(RS, HI + 1 - y0);
  const int wxA = 2 * j + OA, wxB = 2 * j + (OA ^ 1);
  const bool okA = wxA >= LO && wxA <= HI && ox + wxA >= 0 && ox + wxA < m;
  const bool okB = wxB >= LO && wxB <= HI && ox + wxB >= 0 && ox + wxB < m;
  const bool rows_in = oy + y0 >= 0 && oy + y0 + nrows <= m;
  const C* po = U + (1 - COLOUR) * PL + y0 * P + j;
  C* pc = U + COLOUR * PL + y0 * P + j;
  C* pb = B + COLOUR * PL + y0 * P + j;
  C xA = zero_c<T>(), xB = zero_c<T>();
  if constexpr (G1 && formed_coef<T>()) {
    xA = X[OA * HS + j];
    xB = X[(OA ^ 1) * HS + j];
  }
  // formed diagonal: D0 = 4c - k^2
  C D0 = zero_c<T>();
  if constexpr (formed_coef<T>()) D0 = make_float2(__fmaf_rn(4.f, c.x, -K.k2), __fmul_rn(4.f, c.y));
  C up = po[-P], mid = po[0];
#pragma unroll
  for (int r = 0; r < RS; ++r) {
    if (r >= nrows) break;
    const C dn = po[(r + 1) * P];
    const int o = OA ^ (r & 1);
    bool ok = (r & 1) ? okB : okA;
    if (!rows_in) ok = ok && oy + y0 + r >= 0 && oy + y0 + r < m;
    if (ok) {
      const C side = po[r * P + 2 * o - 1];
      const C s = xadd(xadd(xadd(o ? mid : side, o ? side : mid), up), dn);
      C d;
      if constexpr (formed_coef<T>()) {
        if constexpr (G1) d = xfms(D0, (r & 1) ? xB : xA, X[2 * HS + y0 + r]);
        else d = formed_diag<W>(K, D0, X, o, j, y0 + r);
      }
      if constexpr (RESID) {
        if constexpr (!formed_coef<T>()) d = xsub(xscale(c, (T)4), K.q[(long long)(oy + y0 + r) * m + ox + 2 * j + o]);
        pb[r * P] = xfma(xfms(pb[r * P], d, pc[r * P]), c, s);          // b - d u + c s
      } else {
        C di;
        if constexpr (formed_coef<T>()) di = crecip(d);
        else di = X[COLOUR * PL + (y0 + r) * P + j];
        pc[r * P] = xmul(di, xfma(pb[r * P], c, s));                    // d^{-1} (b + c s)
      }
    }
    up = mid;
    mid = dn;
  }
}

// down tile (P0x, P0y in coarse points).  u_in is ignored when zero_init.
// The window origin has ox + oy even, so window colour 0 is red ((fx + fy) even).
template <typename T, int TC, bool COH, bool G1>
__device__ void down_tile(int P0x, int P0y, const cx<T>* u_in, int zero_init, const cx<T>* b,
                          const LevelCoef<T>& K, cx<T> c, int m, int mc, cx<T>* u_out, cx<T>* bc,
                          unsigned char* smem_raw) {
  using C = cx<T>;
  using L = RB<Geo<TC>::DW, (int)sizeof(C)>;
  constexpr int FT = Geo<TC>::FT, DW = Geo<TC>::DW, HS = L::HS, P = L::P, NW = L::ELEMS;
  C* U = reinterpret_cast<C*>(smem_raw);
  C* B = U + NW;                              // RHS, then the red residual in place
  C* X = B + NW;                              // coefficient windows
  const int ox = 2 * P0x - 3, oy = 2 * P0y - 3;   // window origin (fine interior index)
  load_window<T, DW, COH>(ox, oy, m, u_in, zero_init != 0, b, K, U, B, X);
  __syncthreads();
  // red on window [1, DW-2], black on [2, DW-3]
  rb_pass<T, DW, 0, 1, DW - 2, false, G1>(ox, oy, m, K, c, U, B, X);
  __syncthreads();
  rb_pass<T, DW, 1, 2, DW - 3, false, G1>(ox, oy, m, K, c, U, B, X);
  __syncthreads();
  // owned fine points [2P0, 2P0+FT) per axis (the last tile also the final
  // index), the black ones only: the up tile of this level reads no red value
  {
    constexpr int PL = L::PLANE;
    const int ex = (P0x + TC >= mc) ? m : 2 * P0x + FT;
    const int ey = (P0y + TC >= mc) ? m : 2 * P0y + FT;
    // each thread one slot column, rows an even stride apart (fixed colour,
    // constant address steps)
    constexpr int RS = (NT / HS) & ~1;
    const int r0 = threadIdx.x / HS, j = threadIdx.x - r0 * HS;
    const int wx = 2 * j + (((r0 + 3) & 1) ^ 1);
    const int fx = ox + wx;
    if (r0 < RS && wx >= 3 && fx < ex && fx < m) {
      const C* src = U + PL + (r0 + 3) * P + j;
      cx<T>* dst = u_out + (long long)(oy + r0 + 3) * m + fx;
#pragma unroll
      for (int k = 0; k < (FT + 1 + RS - 1) / RS; ++k) {
        const int ly = r0 + k * RS, fy = oy + ly + 3;
        if (ly <= FT && fy < ey && fy < m) *dst = *src;
        src += RS * P;
        dst += (long long)RS * m;
      }
    }
  }
  // residual at the red points of [2P0, 2P0+FT]^2 (window [3, 3+FT]).  At the
  // black points it is zero: the black half sweep has just solved their
  // equations with the final red values.
  rb_pass<T, DW, 0, 3, 3 + FT, true, G1>(ox, oy, m, K, c, U, B, X);
  __syncthreads();
  if constexpr (!COH) pdl_trigger();
  // full weighting: coarse P has its centre fine point 2P+1 at window
  // (2p+4, 2p+4) and corners at (2p+3 | 2p+5, 2p+3 | 2p+5), all red (slots
  // p+2 and p+1, p+2); the four edge points are black, with zero residual
  const C* R0 = B;
  for (int i = threadIdx.x; i < TC * TC; i += NT) {
    const int py = i / TC, px = i - py * TC;
    const int Px = P0x + px, Py = P0y + py;
    if (Px >= mc || Py >= mc) continue;
    const C* r3 = R0 + (2 * py + 3) * P + px;
    const C* r4 = r3 + P;
    const C* r5 = r4 + P;
    const C top = xadd(xscale(r3[1], (T)0.25), xscale(r3[2], (T)0.25));
    const C cen = xscale(r4[2], (T)0.5);
    const C bot = xadd(xscale(r5[1], (T)0.25), xscale(r5[2], (T)0.25));
    bc[(long long)Py * mc + Px] = xadd(xadd(xscale(top, (T)0.25), xscale(cen, (T)0.5)), xscale(bot, (T)0.25));
  }
  __syncthreads();   // shared memory is reused by the next tile
}

// Linear interpolation along one axis from a coarse window whose first entry
// is coarse interior index e0 (coarse values outside [0, mc) are zero).
template <typename T>
__device__ __forceinline__ int interp_w(int p, int e0, int mc, int* ci, T* w) {
  int i = p + 1, n = 0;
  if ((i & 1) == 0) {
    int I = i >> 1;
    if (I >= 1 && I <= mc) { ci[n] = I - 1 - e0; w[n] = (T)1; ++n; }
  } else {
    int I0 = (i - 1) >> 1, I1 = I0 + 1;
    if (I0 >= 1 && I0 <= mc) { ci[n] = I0 - 1 - e0; w[n] = (T)0.5; ++n; }
    if (I1 >= 1 && I1 <= mc) { ci[n] = I1 - 1 - e0; w[n] = (T)0.5; ++n; }
  }
  return n;
}

// up tile: u = u_in + P e_c, one RB-GS sweep, write owned points.  Window
// colour 0 is red (ox + oy even).  In the per-level kernel the tile itself
// waits for the kernel before it (which writes only e_c), after issuing the
// copies of its fine window; the persistent kernel's grid barrier orders it.
template <typename T, int TC, bool COH, bool G1>
__device__ void up_tile(int P0x, int P0y, const cx<T>* u_in, const cx<T>* ec, const cx<T>* b,
                        const LevelCoef<T>& K, cx<T> c, int m, int mc, cx<T>* u_out, unsigned char* smem_raw) {
  using C = cx<T>;
  using L = RB<Geo<TC>::UW, (int)sizeof(C)>;
  constexpr int FT = Geo<TC>::FT, UW = Geo<TC>::UW, EW = Geo<TC>::EW, NW = L::ELEMS;
  C* U = reinterpret_cast<C*>(smem_raw);
  C* B = U + NW;
  C* E = B + NW;                         // EW x EW coarse window
  C* X = E + EW * EW;                    // coefficient windows
  const int ox = 2 * P0x - 2, oy = 2 * P0y - 2;
  const int ex0 = P0x - 2, ey0 = P0y - 2;
  // per-level kernels: the window copies go out before the wait for the
  // predecessor, which writes only the coarse correction
  if constexpr (!COH) {
    load_window<T, UW, COH, false>(ox, oy, m, u_in, false, b, K, U, B, X);
    pdl_prologue();
  }
  // coarse window: asynchronous copies (per-level kernels) or loads held in
  // registers across the fine window's loads (persistent kernel)
  constexpr int NKE = (EW * EW + NT - 1) / NT;
  C ev[NKE];
#pragma unroll
  for (int k = 0; k < NKE; ++k) {
    const int i = threadIdx.x + k * NT;
    const int wy = i / EW, wx = i - wy * EW;
    const int cxp = ex0 + wx, cyp = ey0 + wy;
    const bool in = i < EW * EW && cxp >= 0 && cxp < mc && cyp >= 0 && cyp < mc;
    if constexpr (COH) ev[k] = in ? ld<COH>(ec + (cyp * mc + cxp)) : zero_c<T>();
    else if (i < EW * EW) cp_async_sz<(int)sizeof(C)>(smem_addr(E + i), ec + (in ? cyp * mc + cxp : 0), in);
  }
  if constexpr (COH) {
    load_window<T, UW, COH>(ox, oy, m, u_in, false, b, K, U, B, X);
#pragma unroll
    for (int k = 0; k < NKE; ++k)
      if (threadIdx.x + k * NT < EW * EW) E[threadIdx.x + k * NT] = ev[k];
  } else {
    cp_async_wait_all();
  }
  __syncthreads();
  // prolongation at the black points only: the red half sweep overwrites the
  // red ones without reading them.  With node index i = f + 1, a black fine
  // point has one odd and one even index: in odd window rows (iy even) it lies
  // between coarse-window columns j and j+1 of row (wy+1)/2, in even rows (iy
  // odd) between rows wy/2 and wy/2+1 of column j+1.  The coarse window is
  // zero outside the coarse interior, so points outside the domain stay zero.
  // Each thread takes slot column j of the black plane and rows an even
  // stride apart, so the row parity, the coarse neighbours' layout and every
  // address step are fixed for the thread.  u + (e0 + e1)/2 as one fused
  // multiply-add: the halving is exact, so this rounds like u + e0/2 + e1/2
  // summed as (e0/2 + e1/2) first.
  {
    constexpr int HS = L::HS, P = L::P, PL = L::PLANE;
    constexpr int RS = (NT / HS) & ~1, NK = (UW + RS - 1) / RS;
    const int r0 = threadIdx.x / HS, j = threadIdx.x - r0 * HS;
    const bool odd = r0 & 1;
    if (r0 < RS && 2 * j + (odd ? 0 : 1) < UW) {
      const C* e = odd ? E + ((r0 + 1) >> 1) * EW + j : E + (r0 >> 1) * EW + j + 1;
      const int e1 = odd ? 1 : EW;
      C* uu = U + PL + r0 * P + j;
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        if (r0 + k * RS < UW) {
          const C* ek = e + k * (RS / 2) * EW;
          uu[k * RS * P] = xfma_r(uu[k * RS * P], xadd(ek[0], ek[e1]), (T)0.5);
        }
      }
    }
  }
  __syncthreads();
  rb_pass<T, UW, 0, 1, UW - 2, false, G1>(ox, oy, m, K, c, U, B, X);
  __syncthreads();
  rb_pass<T, UW, 1, 2, UW - 3, false, G1>(ox, oy, m, K, c, U, B, X);
  __syncthreads();
  if constexpr (!COH) pdl_trigger();
  const int exx = (P0x + TC >= mc) ? m : 2 * P0x + FT;
  const int eyy = (P0y + TC >= mc) ? m : 2 * P0y + FT;
  {
    // each thread one column, rows an even stride apart (fixed colour,
    // constant address steps)
    constexpr int RS = (NT / (FT + 1)) & ~1;
    const int r0 = threadIdx.x / (FT + 1), lx = threadIdx.x - r0 * (FT + 1);
    const int fx = 2 * P0x + lx;
    if (r0 < RS && fx < exx && fx < m) {
      const C* src = U + rbi<UW, (int)sizeof(C)>(lx + 2, r0 + 2);
      cx<T>* dst = u_out + (long long)(2 * P0y + r0) * m + fx;
#pragma unroll
      for (int k = 0; k < (FT + 1 + RS - 1) / RS; ++k) {
        const int ly = r0 + k * RS, fy = 2 * P0y + ly;
        if (ly <= FT && fy < eyy && fy < m) *dst = *src;
        src += RS * L::P;
        dst += (long long)RS * m;
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// All levels from lc down to the coarsest and back in one CTA.  Level data
// (u, b, r and the coefficients) lives in shared memory.
// ---------------------------------------------------------------------------
struct CoarseLevels {
  int nl;                       // number of levels handled (last = coarsest)
  int m[8];
  const void* q[8];
  const void* dinv[8];
  double2 c[8];
  float2 c32[8];                // c rounded to FP32 (FP32 cycles)
};

template <typename T> __device__ __forceinline__ cx<T> level_c(const CoarseLevels& L, int l);
template <> __device__ __forceinline__ double2 level_c<double>(const CoarseLevels& L, int l) { return L.c[l]; }
template <> __device__ __forceinline__ float2 level_c<float>(const CoarseLevels& L, int l) { return L.c32[l]; }

template <typename T, int D>
__device__ __forceinline__ cx<T> apply_s(const cx<T>* u, int m, int ix, int iy, int iz, int idx, cx<T> q,
                                         cx<T> c) {
  using C = cx<T>;
  C s = zero_c<T>();
  if (ix > 0) s = xadd(s, u[idx - 1]);
  if (ix < m - 1) s = xadd(s, u[idx + 1]);
  if (iy > 0) s = xadd(s, u[idx - m]);
  if (iy < m - 1) s = xadd(s, u[idx + m]);
  if (D == 3) {
    if (iz > 0) s = xadd(s, u[idx - m * m]);
    if (iz < m - 1) s = xadd(s, u[idx + m * m]);
  }
  C uj = u[idx];
  C t = xsub(xscale(uj, (T)(2 * D)), s);
  return xsub(xmul(c, t), xmul(q, uj));
}

template <int D>
__device__ __forceinline__ void decode(int i, int m, int& ix, int& iy, int& iz) {
  ix = i % m;
  int r = i / m;
  if (D == 3) { iy = r % m; iz = r / m; } else { iy = r; iz = 0; }
}

template <typename T, int D>
__device__ void rbgs_s(cx<T>* u, const cx<T>* b, const cx<T>* q, const cx<T>* dinv, cx<T> c, int m, int N) {
  for (int colour = 0; colour < 2; ++colour) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      int ix, iy, iz;
      decode<D>(i, m, ix, iy, iz);
      if (((ix + iy + iz + D) & 1) != colour) continue;
      cx<T> rj = xsub(b[i], apply_s<T, D>(u, m, ix, iy, iz, i, q[i], c));
      u[i] = xadd(u[i], xmul(dinv[i], rj));
    }
    __syncthreads();
  }
}

inline size_t coarse_levels_elems(const std::vector<Level>& lv, int lc) {
  size_t n = 0;
  for (size_t l = lc; l < lv.size(); ++l) n += 5 * (size_t)lv[l].N;
  return n;
}

template <typename T> __device__ __forceinline__ cx<T> to_cx(double2 v);
template <> __device__ __forceinline__ double2 to_cx<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 to_cx<float>(double2 v) {
  return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
}
template <typename TI, typename T> __device__ __forceinline__ cx<TI> widen(cx<T> v) {
  return mk<cx<TI>>((TI)v.x, (TI)v.y);
}

// TI: the arithmetic of the coarsest product (T, or double for FP32 cycles
// whose coarsest solve runs in FP64; the product is then rounded to T once)
template <typename T, int D, bool COH, typename TI = T>
__device__ void coarse_levels_block(const CoarseLevels& L, const cx<T>* b_top, cx<T>* u_top,
                                    const cx<TI>* __restrict__ inv, unsigned char* smem_raw) {
  using C = cx<T>;
  C* base = reinterpret_cast<C*>(smem_raw);
  C* U[8];
  C* B[8];
  C* R[8];
  C* Qs[8];
  C* Ds[8];
  int N[8];
  {
    C* p = base;
    for (int l = 0; l < L.nl; ++l) {
      N[l] = L.m[l] * L.m[l] * (D == 3 ? L.m[l] : 1);
      U[l] = p; p += N[l];
      B[l] = p; p += N[l];
      R[l] = p; p += N[l];
      Qs[l] = p; p += N[l];
      Ds[l] = p; p += N[l];
    }
  }
  // every global read up front; the phases below touch shared memory only.
  // Each thread's first point of every level is loaded into registers before
  // any store, so those loads are in flight together; the rest follow.
  {
    const int t = threadIdx.x;
    C qv[8], dv[8];
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l < L.nl && t < N[l]) {
        qv[l] = reinterpret_cast<const C*>(L.q[l])[t];
        dv[l] = reinterpret_cast<const C*>(L.dinv[l])[t];
      }
    const C bv = (t < N[0]) ? ld<COH>(b_top + t) : zero_c<T>();
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (l < L.nl && t < N[l]) {
        Qs[l][t] = qv[l];
        Ds[l][t] = dv[l];
      }
    if (t < N[0]) {
      B[0][t] = bv;
      U[0][t] = zero_c<T>();
    }
  }
  for (int l = 0; l < L.nl; ++l) {
    const C* q = reinterpret_cast<const C*>(L.q[l]);
    const C* dv = reinterpret_cast<const C*>(L.dinv[l]);
    for (int i = threadIdx.x + blockDim.x; i < N[l]; i += blockDim.x) {
      Qs[l][i] = q[i];
      Ds[l][i] = dv[i];
    }
  }
  for (int i = threadIdx.x + blockDim.x; i < N[0]; i += blockDim.x) {
    B[0][i] = ld<COH>(b_top + i);
    U[0][i] = zero_c<T>();
  }
  __syncthreads();
  const T w1[3] = {(T)0.25, (T)0.5, (T)0.25};
  const int last = L.nl - 1;
  for (int l = 0; l < last; ++l) {
    const int m = L.m[l], mc = L.m[l + 1];
    const C c = level_c<T>(L, l);
    if (l > 0)
      for (int i = threadIdx.x; i < N[l]; i += blockDim.x) U[l][i] = zero_c<T>();
    __syncthreads();
    rbgs_s<T, D>(U[l], B[l], Qs[l], Ds[l], c, m, N[l]);
    for (int i = threadIdx.x; i < N[l]; i += blockDim.x) {
      int ix, iy, iz;
      decode<D>(i, m, ix, iy, iz);
      R[l][i] = xsub(B[l][i], apply_s<T, D>(U[l], m, ix, iy, iz, i, Qs[l][i], c));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N[l + 1]; i += blockDim.x) {
      int px, py, pz;
      decode<D>(i, mc, px, py, pz);
      C acc = zero_c<T>();
      for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            int fx = 2 * px + 1 + ox, fy = 2 * py + 1 + oy, fz = (D == 3) ? 2 * pz + 1 + oz : 0;
            T w = w1[ox + 1] * w1[oy + 1] * ((D == 3) ? w1[oz + 1] : (T)1);
            acc = xadd(acc, xscale(R[l][(fz * m + fy) * m + fx], w));
          }
      B[l + 1][i] = acc;
    }
    __syncthreads();
  }
  // coarsest: u = inv b (the inverse itself comes from FP64 Gauss-Jordan)
  if constexpr (sizeof(TI) == sizeof(T)) {
    // in the cycle's precision: one warp per row, lanes split the columns
    const int n = N[last];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < n; i += nw) {
      C acc = zero_c<T>();
      const C* row = inv + (long long)i * n;
      for (int j = lane; j < n; j += 32) acc = xadd(acc, xmul(row[j], B[last][j]));
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) U[last][i] = acc;
    }
    __syncthreads();
  } else {
    // in FP64 (FP32 cycles of the FP64 refinement): FP64 work is scarce, so
    // each row is split over four consecutive lanes only (columns j = p mod 4),
    // each lane a chain of fused multiply-adds; two shuffles join the parts and
    // the row's sum is rounded once to the cycle's precision
    const int n = N[last];
    for (int t = threadIdx.x; t < ((4 * n + 31) & ~31); t += blockDim.x) {
      const int i = t >> 2, part = t & 3;
      double re = 0.0, im = 0.0;
      if (i < n) {
        const double2* row = reinterpret_cast<const double2*>(inv) + (long long)i * n;
        for (int j = part; j < n; j += 4) {
          const double2 a = row[j];
          const double bx = (double)B[last][j].x, by = (double)B[last][j].y;
          re = fma(a.x, bx, fma(-a.y, by, re));
          im = fma(a.x, by, fma(a.y, bx, im));
        }
      }
      re += __shfl_xor_sync(0xffffffffu, re, 1);
      im += __shfl_xor_sync(0xffffffffu, im, 1);
      re += __shfl_xor_sync(0xffffffffu, re, 2);
      im += __shfl_xor_sync(0xffffffffu, im, 2);
      if (i < n && part == 0) U[last][i] = to_cx<T>(make_double2(re, im));
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= 0; --l) {
    const int m = L.m[l], mc = L.m[l + 1];
    const C c = level_c<T>(L, l);
    for (int i = threadIdx.x; i < N[l]; i += blockDim.x) {
      int ix, iy, iz;
      decode<D>(i, m, ix, iy, iz);
      int cxi[2], cyi[2], czi[2] = {0, 0};
      T wx[2], wy[2], wz[2] = {(T)1, (T)0};
      int nx = interp_w<T>(ix, 0, mc, cxi, wx);
      int ny = interp_w<T>(iy, 0, mc, cyi, wy);
      int nz = (D == 3) ? interp_w<T>(iz, 0, mc, czi, wz) : 1;
      C acc = zero_c<T>();
      for (int a = 0; a < nz; ++a)
        for (int bq = 0; bq < ny; ++bq)
          for (int cq = 0; cq < nx; ++cq)
            acc = xadd(acc, xscale(U[l + 1][(czi[a] * mc + cyi[bq]) * mc + cxi[cq]], wx[cq] * wy[bq] * wz[a]));
      U[l][i] = xadd(U[l][i], acc);
    }
    __syncthreads();
    rbgs_s<T, D>(U[l], B[l], Qs[l], Ds[l], c, m, N[l]);
  }
  for (int i = threadIdx.x; i < N[0]; i += blockDim.x) u_top[i] = U[0][i];
  __syncthreads();
}

}  // namespace tiles
}  // namespace csff
