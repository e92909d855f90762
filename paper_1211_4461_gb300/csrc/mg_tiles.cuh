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

template <int TC> __host__ __device__ constexpr size_t down_smem_elems() {
  return (size_t)(4 * Geo<TC>::DW * Geo<TC>::DW + (Geo<TC>::FT + 1) * (Geo<TC>::FT + 1));
}
template <int TC> __host__ __device__ constexpr size_t up_smem_elems() {
  return (size_t)(4 * Geo<TC>::UW * Geo<TC>::UW + Geo<TC>::EW * Geo<TC>::EW);
}

template <typename T>
__device__ __forceinline__ cx<T> zero_c() { return mk<cx<T>>((T)0, (T)0); }

template <bool COH, typename C>
__device__ __forceinline__ C ld(const C* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// A u at window point (wy, wx) of a row-major window of width W (values
// outside the domain are stored as zero).  Neighbour order x-1, x+1, y-1, y+1
// as in the unfused kernels.
template <typename T>
__device__ __forceinline__ cx<T> apply_w(const cx<T>* U, int W, int wy, int wx, cx<T> q, cx<T> c) {
  using C = cx<T>;
  C uj = U[wy * W + wx];
  C s = cadd(cadd(cadd(U[wy * W + wx - 1], U[wy * W + wx + 1]), U[(wy - 1) * W + wx]), U[(wy + 1) * W + wx]);
  C t = csub(cscale(uj, (T)4), s);
  return csub(cmul(c, t), cmul(q, uj));
}

// down tile (P0x, P0y in coarse points).  u_in is ignored when zero_init.
template <typename T, int TC, bool COH>
__device__ void down_tile(int P0x, int P0y, const cx<T>* u_in, int zero_init, const cx<T>* b,
                          const cx<T>* __restrict__ q, const cx<T>* __restrict__ dinv, cx<T> c, int m, int mc,
                          cx<T>* u_out, cx<T>* bc, unsigned char* smem_raw) {
  using C = cx<T>;
  constexpr int FT = Geo<TC>::FT, DW = Geo<TC>::DW;
  C* U = reinterpret_cast<C*>(smem_raw);
  C* B = U + DW * DW;
  C* Q = B + DW * DW;
  C* Dv = Q + DW * DW;
  C* R = Dv + DW * DW;                   // residual on fine [2P0, 2P0+2TC], (FT+1)^2
  const int ox = 2 * P0x - 3, oy = 2 * P0y - 3;   // window origin (fine interior index)
  for (int i = threadIdx.x; i < DW * DW; i += NT) {
    int wy = i / DW, wx = i - wy * DW;
    int fx = ox + wx, fy = oy + wy;
    bool in = fx >= 0 && fx < m && fy >= 0 && fy < m;
    long long g = (long long)fy * m + fx;
    U[i] = (in && !zero_init) ? ld<COH>(u_in + g) : zero_c<T>();
    B[i] = in ? ld<COH>(b + g) : zero_c<T>();
    Q[i] = in ? q[g] : zero_c<T>();
    Dv[i] = in ? dinv[g] : zero_c<T>();
  }
  __syncthreads();
  // red on window [1, DW-2], black on [2, DW-3]; colour from the node-index sum
  for (int colour = 0; colour < 2; ++colour) {
    const int lo = 1 + colour, hi = DW - 2 - colour;
    for (int i = threadIdx.x; i < DW * DW; i += NT) {
      int wy = i / DW, wx = i - wy * DW;
      if (wx < lo || wx > hi || wy < lo || wy > hi) continue;
      int fx = ox + wx, fy = oy + wy;
      if (fx < 0 || fx >= m || fy < 0 || fy >= m) continue;
      if (((fx + fy) & 1) != colour) continue;
      C rj = csub(B[i], apply_w<T>(U, DW, wy, wx, Q[i], c));
      U[i] = cadd(U[i], cmul(Dv[i], rj));
    }
    __syncthreads();
  }
  // owned fine points: [2P0, 2P0+FT) per axis, the last tile also the final index
  {
    const int ex = (P0x + TC >= mc) ? m : 2 * P0x + FT;
    const int ey = (P0y + TC >= mc) ? m : 2 * P0y + FT;
    for (int i = threadIdx.x; i < (FT + 1) * (FT + 1); i += NT) {
      int ly = i / (FT + 1), lx = i - ly * (FT + 1);
      int fx = 2 * P0x + lx, fy = 2 * P0y + ly;
      int wx = lx + 3, wy = ly + 3;
      if (fx < ex && fy < ey && fx < m && fy < m) u_out[(long long)fy * m + fx] = U[wy * DW + wx];
      C rv = zero_c<T>();
      if (fx < m && fy < m) rv = csub(B[wy * DW + wx], apply_w<T>(U, DW, wy, wx, Q[wy * DW + wx], c));
      R[i] = rv;
    }
  }
  __syncthreads();
  const T w1[3] = {(T)0.25, (T)0.5, (T)0.25};
  for (int i = threadIdx.x; i < TC * TC; i += NT) {
    int py = i / TC, px = i - py * TC;
    int Px = P0x + px, Py = P0y + py;
    if (Px >= mc || Py >= mc) continue;
    C acc = zero_c<T>();
#pragma unroll
    for (int oy2 = -1; oy2 <= 1; ++oy2) {
      C row = zero_c<T>();
      int ry = 2 * py + 1 + oy2;
#pragma unroll
      for (int ox2 = -1; ox2 <= 1; ++ox2) row = cadd(row, cscale(R[ry * (FT + 1) + 2 * px + 1 + ox2], w1[ox2 + 1]));
      acc = cadd(acc, cscale(row, w1[oy2 + 1]));
    }
    bc[(long long)Py * mc + Px] = acc;
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

// up tile: u = u_in + P e_c, one RB-GS sweep, write owned points.
template <typename T, int TC, bool COH>
__device__ void up_tile(int P0x, int P0y, const cx<T>* u_in, const cx<T>* ec, const cx<T>* b,
                        const cx<T>* __restrict__ q, const cx<T>* __restrict__ dinv, cx<T> c, int m, int mc,
                        cx<T>* u_out, unsigned char* smem_raw) {
  using C = cx<T>;
  constexpr int FT = Geo<TC>::FT, UW = Geo<TC>::UW, EW = Geo<TC>::EW;
  C* U = reinterpret_cast<C*>(smem_raw);
  C* B = U + UW * UW;
  C* Q = B + UW * UW;
  C* Dv = Q + UW * UW;
  C* E = Dv + UW * UW;                   // EW x EW coarse window
  const int ox = 2 * P0x - 2, oy = 2 * P0y - 2;
  const int ex0 = P0x - 2, ey0 = P0y - 2;
  for (int i = threadIdx.x; i < EW * EW; i += NT) {
    int wy = i / EW, wx = i - wy * EW;
    int cxp = ex0 + wx, cyp = ey0 + wy;
    E[i] = (cxp >= 0 && cxp < mc && cyp >= 0 && cyp < mc) ? ld<COH>(ec + (long long)cyp * mc + cxp) : zero_c<T>();
  }
  for (int i = threadIdx.x; i < UW * UW; i += NT) {
    int wy = i / UW, wx = i - wy * UW;
    int fx = ox + wx, fy = oy + wy;
    bool in = fx >= 0 && fx < m && fy >= 0 && fy < m;
    long long g = (long long)fy * m + fx;
    U[i] = in ? ld<COH>(u_in + g) : zero_c<T>();
    B[i] = in ? ld<COH>(b + g) : zero_c<T>();
    Q[i] = in ? q[g] : zero_c<T>();
    Dv[i] = in ? dinv[g] : zero_c<T>();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < UW * UW; i += NT) {
    int wy = i / UW, wx = i - wy * UW;
    int fx = ox + wx, fy = oy + wy;
    if (fx < 0 || fx >= m || fy < 0 || fy >= m) continue;
    int cxi[2], cyi[2];
    T wxs[2], wys[2];
    int nx = interp_w<T>(fx, ex0, mc, cxi, wxs);
    int ny = interp_w<T>(fy, ey0, mc, cyi, wys);
    C acc = zero_c<T>();
    for (int a = 0; a < ny; ++a)
      for (int bb = 0; bb < nx; ++bb) acc = cadd(acc, cscale(E[cyi[a] * EW + cxi[bb]], wxs[bb] * wys[a]));
    U[i] = cadd(U[i], acc);
  }
  __syncthreads();
  for (int colour = 0; colour < 2; ++colour) {
    const int lo = 1 + colour, hi = UW - 2 - colour;
    for (int i = threadIdx.x; i < UW * UW; i += NT) {
      int wy = i / UW, wx = i - wy * UW;
      if (wx < lo || wx > hi || wy < lo || wy > hi) continue;
      int fx = ox + wx, fy = oy + wy;
      if (fx < 0 || fx >= m || fy < 0 || fy >= m) continue;
      if (((fx + fy) & 1) != colour) continue;
      C rj = csub(B[i], apply_w<T>(U, UW, wy, wx, Q[i], c));
      U[i] = cadd(U[i], cmul(Dv[i], rj));
    }
    __syncthreads();
  }
  const int exx = (P0x + TC >= mc) ? m : 2 * P0x + FT;
  const int eyy = (P0y + TC >= mc) ? m : 2 * P0y + FT;
  for (int i = threadIdx.x; i < (FT + 1) * (FT + 1); i += NT) {
    int ly = i / (FT + 1), lx = i - ly * (FT + 1);
    int fx = 2 * P0x + lx, fy = 2 * P0y + ly;
    if (fx < exx && fy < eyy && fx < m && fy < m) u_out[(long long)fy * m + fx] = U[(ly + 2) * UW + lx + 2];
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
};

template <typename T, int D>
__device__ __forceinline__ cx<T> apply_s(const cx<T>* u, int m, int ix, int iy, int iz, int idx, cx<T> q,
                                         cx<T> c) {
  using C = cx<T>;
  C s = zero_c<T>();
  if (ix > 0) s = cadd(s, u[idx - 1]);
  if (ix < m - 1) s = cadd(s, u[idx + 1]);
  if (iy > 0) s = cadd(s, u[idx - m]);
  if (iy < m - 1) s = cadd(s, u[idx + m]);
  if (D == 3) {
    if (iz > 0) s = cadd(s, u[idx - m * m]);
    if (iz < m - 1) s = cadd(s, u[idx + m * m]);
  }
  C uj = u[idx];
  C t = csub(cscale(uj, (T)(2 * D)), s);
  return csub(cmul(c, t), cmul(q, uj));
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
      cx<T> rj = csub(b[i], apply_s<T, D>(u, m, ix, iy, iz, i, q[i], c));
      u[i] = cadd(u[i], cmul(dinv[i], rj));
    }
    __syncthreads();
  }
}

inline size_t coarse_levels_elems(const std::vector<Level>& lv, int lc) {
  size_t n = 0;
  for (size_t l = lc; l < lv.size(); ++l) n += 5 * (size_t)lv[l].N;
  return n;
}

template <typename T, int D, bool COH>
__device__ void coarse_levels_block(const CoarseLevels& L, const cx<T>* b_top, cx<T>* u_top,
                                    const cx<T>* __restrict__ inv, unsigned char* smem_raw) {
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
  // every global read up front (independent loads in flight together); the
  // phases below touch shared memory only
  for (int l = 0; l < L.nl; ++l) {
    const C* q = reinterpret_cast<const C*>(L.q[l]);
    const C* dv = reinterpret_cast<const C*>(L.dinv[l]);
    for (int i = threadIdx.x; i < N[l]; i += blockDim.x) {
      Qs[l][i] = q[i];
      Ds[l][i] = dv[i];
    }
  }
  for (int i = threadIdx.x; i < N[0]; i += blockDim.x) {
    B[0][i] = ld<COH>(b_top + i);
    U[0][i] = zero_c<T>();
  }
  __syncthreads();
  const T w1[3] = {(T)0.25, (T)0.5, (T)0.25};
  const int last = L.nl - 1;
  for (int l = 0; l < last; ++l) {
    const int m = L.m[l], mc = L.m[l + 1];
    C c = mk<C>((T)L.c[l].x, (T)L.c[l].y);
    if (l > 0)
      for (int i = threadIdx.x; i < N[l]; i += blockDim.x) U[l][i] = zero_c<T>();
    __syncthreads();
    rbgs_s<T, D>(U[l], B[l], Qs[l], Ds[l], c, m, N[l]);
    for (int i = threadIdx.x; i < N[l]; i += blockDim.x) {
      int ix, iy, iz;
      decode<D>(i, m, ix, iy, iz);
      R[l][i] = csub(B[l][i], apply_s<T, D>(U[l], m, ix, iy, iz, i, Qs[l][i], c));
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
            acc = cadd(acc, cscale(R[l][(fz * m + fy) * m + fx], w));
          }
      B[l + 1][i] = acc;
    }
    __syncthreads();
  }
  // coarsest: u = inv b in the cycle's precision (the inverse itself comes from
  // FP64 Gauss-Jordan), one warp per row, lanes split the columns
  {
    const int n = N[last];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < n; i += nw) {
      C acc = zero_c<T>();
      const C* row = inv + (long long)i * n;
      for (int j = lane; j < n; j += 32) acc = cadd(acc, cmul(row[j], B[last][j]));
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) U[last][i] = acc;
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= 0; --l) {
    const int m = L.m[l], mc = L.m[l + 1];
    C c = mk<C>((T)L.c[l].x, (T)L.c[l].y);
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
            acc = cadd(acc, cscale(U[l + 1][(czi[a] * mc + cyi[bq]) * mc + cxi[cq]], wx[cq] * wy[bq] * wz[a]));
      U[l][i] = cadd(U[l][i], acc);
    }
    __syncthreads();
    rbgs_s<T, D>(U[l], B[l], Qs[l], Ds[l], c, m, N[l]);
  }
  for (int i = threadIdx.x; i < N[0]; i += blockDim.x) u_top[i] = U[0][i];
  __syncthreads();
}

}  // namespace tiles
}  // namespace csff
