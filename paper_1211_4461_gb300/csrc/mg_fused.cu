// Fused V(1,1) red-black Gauss-Seidel multigrid kernels (2D).
//
// The V-cycle of Sec. 4 with one red-black sweep before and after the
// coarse-grid correction is executed as
//   down(l):  RB-GS sweep on A_l u = b_l, r = b_l - A_l u, b_{l+1} = FW(r)
//   coarse:   every level from lc to the coarsest in one CTA (shared memory)
//   up(l):    u += P u_{l+1}, RB-GS sweep
// Each down/up kernel reads a tile of the fine grid plus a halo into shared
// memory once (halo 3 for down: red update on the tile+2, black on tile+1,
// residual on the tile; halo 2 for up), so one level costs two passes over
// its arrays instead of eight kernels.  The smoothed iterate of down(l) goes to
// a second buffer (the halos of neighbouring tiles must see the old values);
// up(l) reads it and writes the final iterate back.  Arithmetic is identical
// to the unfused kernels (same operation order per point).
#include "csff_internal.h"

namespace csff {
namespace {

// Tile geometry for TC coarse points per tile side: the tile owns FT = 2 TC
// fine points per side; down window fine [2P0-3, 2P0+2TC+3], up window fine
// [2P0-2, 2P0+2TC+2], coarse window for up [P0-2, P0+TC+1].  Large levels use
// TC = 16; levels with few tiles use TC = 8 (shorter per-block latency).
template <int TC> struct Geo {
  static constexpr int FT = 2 * TC;
  static constexpr int DW = FT + 7;
  static constexpr int UW = FT + 5;
  static constexpr int EW = TC + 4;
};
constexpr int NT = 256;

template <typename T>
__device__ __forceinline__ cx<T> zero_c() { return mk<cx<T>>((T)0, (T)0); }

// A u at window point (wy, wx) of a row-major window of width W (values
// outside the domain are stored as zero).
template <typename T>
__device__ __forceinline__ cx<T> apply_w(const cx<T>* U, int W, int wy, int wx, cx<T> q, cx<T> c) {
  using C = cx<T>;
  C uj = U[wy * W + wx];
  C s = cadd(cadd(cadd(U[wy * W + wx - 1], U[wy * W + wx + 1]), U[(wy - 1) * W + wx]), U[(wy + 1) * W + wx]);
  C t = csub(cscale(uj, (T)4), s);
  return csub(cmul(c, t), cmul(q, uj));
}

// down: one RB-GS sweep, residual, full weighting.
template <typename T, int TC>
__global__ void __launch_bounds__(NT) k_down2(const cx<T>* __restrict__ u_in, int zero_init,
                                              const cx<T>* __restrict__ b, const cx<T>* __restrict__ q,
                                              const cx<T>* __restrict__ dinv, cx<T> c, int m, int mc,
                                              cx<T>* __restrict__ u_out, cx<T>* __restrict__ bc) {
  using C = cx<T>;
  constexpr int FT = Geo<TC>::FT, DW = Geo<TC>::DW;
  extern __shared__ unsigned char smem_raw[];
  C* U = reinterpret_cast<C*>(smem_raw);
  C* B = U + DW * DW;
  C* Q = B + DW * DW;
  C* Dv = Q + DW * DW;
  C* R = Dv + DW * DW;                   // residual on fine [2P0, 2P0+2TC], (FT+1)^2
  const int P0x = blockIdx.x * TC, P0y = blockIdx.y * TC;
  const int ox = 2 * P0x - 3, oy = 2 * P0y - 3;   // window origin (fine interior index)
  for (int i = threadIdx.x; i < DW * DW; i += NT) {
    int wy = i / DW, wx = i - wy * DW;
    int fx = ox + wx, fy = oy + wy;
    bool in = fx >= 0 && fx < m && fy >= 0 && fy < m;
    long long g = (long long)fy * m + fx;
    U[i] = (in && !zero_init) ? u_in[g] : zero_c<T>();
    B[i] = in ? b[g] : zero_c<T>();
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
      // residual on [2P0, 2P0+2TC]
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

// up: u = u_in + P e_c, one RB-GS sweep, write owned points.
template <typename T, int TC>
__global__ void __launch_bounds__(NT) k_up2(const cx<T>* __restrict__ u_in, const cx<T>* __restrict__ ec,
                                            const cx<T>* __restrict__ b, const cx<T>* __restrict__ q,
                                            const cx<T>* __restrict__ dinv, cx<T> c, int m, int mc,
                                            cx<T>* __restrict__ u_out) {
  using C = cx<T>;
  constexpr int FT = Geo<TC>::FT, UW = Geo<TC>::UW, EW = Geo<TC>::EW;
  extern __shared__ unsigned char smem_raw[];
  C* U = reinterpret_cast<C*>(smem_raw);
  C* B = U + UW * UW;
  C* Q = B + UW * UW;
  C* Dv = Q + UW * UW;
  C* E = Dv + UW * UW;                   // EW x EW coarse window
  const int P0x = blockIdx.x * TC, P0y = blockIdx.y * TC;
  const int ox = 2 * P0x - 2, oy = 2 * P0y - 2;
  const int ex0 = P0x - 2, ey0 = P0y - 2;
  for (int i = threadIdx.x; i < EW * EW; i += NT) {
    int wy = i / EW, wx = i - wy * EW;
    int cxp = ex0 + wx, cyp = ey0 + wy;
    E[i] = (cxp >= 0 && cxp < mc && cyp >= 0 && cyp < mc) ? ec[(long long)cyp * mc + cxp] : zero_c<T>();
  }
  for (int i = threadIdx.x; i < UW * UW; i += NT) {
    int wy = i / UW, wx = i - wy * UW;
    int fx = ox + wx, fy = oy + wy;
    bool in = fx >= 0 && fx < m && fy >= 0 && fy < m;
    long long g = (long long)fy * m + fx;
    U[i] = in ? u_in[g] : zero_c<T>();
    B[i] = in ? b[g] : zero_c<T>();
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
}

// ---------------------------------------------------------------------------
// All levels from lc down to the coarsest and back in one CTA.  Level data
// (u, b, r) lives in shared memory; coefficients are read from global memory.
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

template <typename T, int D>
__global__ void __launch_bounds__(1024) k_coarse_levels(CoarseLevels L, const cx<T>* __restrict__ b_top,
                                                        cx<T>* __restrict__ u_top, const double2* __restrict__ inv) {
  using C = cx<T>;
  extern __shared__ unsigned char smem_raw[];
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
    B[0][i] = b_top[i];
    U[0][i] = zero_c<T>();
  }
  __syncthreads();
  const T w1[3] = {(T)0.25, (T)0.5, (T)0.25};
  const int last = L.nl - 1;
  // down
  for (int l = 0; l < last; ++l) {
    const int m = L.m[l], mc = L.m[l + 1];
    const C* q = Qs[l];
    const C* dv = Ds[l];
    C c = mk<C>((T)L.c[l].x, (T)L.c[l].y);
    if (l > 0)
      for (int i = threadIdx.x; i < N[l]; i += blockDim.x) U[l][i] = zero_c<T>();
    __syncthreads();
    rbgs_s<T, D>(U[l], B[l], q, dv, c, m, N[l]);
    for (int i = threadIdx.x; i < N[l]; i += blockDim.x) {
      int ix, iy, iz;
      decode<D>(i, m, ix, iy, iz);
      R[l][i] = csub(B[l][i], apply_s<T, D>(U[l], m, ix, iy, iz, i, q[i], c));
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
  // coarsest: u = inv b (FP64)
  {
    const int n = N[last];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double2 acc = make_double2(0, 0);
      const double2* row = inv + (long long)i * n;
      for (int j = 0; j < n; ++j) acc = cadd(acc, cmul(row[j], make_double2((double)B[last][j].x, (double)B[last][j].y)));
      U[last][i] = mk<C>((T)acc.x, (T)acc.y);
    }
    __syncthreads();
  }
  // up
  for (int l = last - 1; l >= 0; --l) {
    const int m = L.m[l], mc = L.m[l + 1];
    const C* q = Qs[l];
    const C* dv = Ds[l];
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
    rbgs_s<T, D>(U[l], B[l], q, dv, c, m, N[l]);
  }
  for (int i = threadIdx.x; i < N[0]; i += blockDim.x) u_top[i] = U[0][i];
}

template <typename T> const cx<T>* qt(const Level& L);
template <> const double2* qt<double>(const Level& L) { return L.q64; }
template <> const float2* qt<float>(const Level& L) { return L.q32; }
template <typename T> const cx<T>* dt(const Level& L);
template <> const double2* dt<double>(const Level& L) { return L.dinv64; }
template <> const float2* dt<float>(const Level& L) { return L.dinv32; }

}  // namespace

template <int TC> size_t down_smem(int rb) {
  return (size_t)(4 * Geo<TC>::DW * Geo<TC>::DW + (Geo<TC>::FT + 1) * (Geo<TC>::FT + 1)) * 2 * rb;
}
template <int TC> size_t up_smem(int rb) {
  return (size_t)(4 * Geo<TC>::UW * Geo<TC>::UW + Geo<TC>::EW * Geo<TC>::EW) * 2 * rb;
}
size_t fused_down_smem(int real_bytes) { return down_smem<16>(real_bytes); }
size_t fused_up_smem(int real_bytes) { return up_smem<16>(real_bytes); }
// tiles of 16 coarse points unless that leaves fewer CTAs than SMs
static bool small_tiles(int mc) { return ((mc + 15) / 16) * ((mc + 15) / 16) < 152; }

template <typename T>
cudaError_t launch_down2(const Level& F, const Level& Cl, const cx<T>* u_in, bool zero_init, const cx<T>* b,
                         cx<T>* u_out, cx<T>* bc, cudaStream_t s) {
  cx<T> c = mk<cx<T>>((T)F.c.x, (T)F.c.y);
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * (3.0 * F.N + Cl.N), 0);
  if (small_tiles(Cl.m)) {
    dim3 g((Cl.m + 7) / 8, (Cl.m + 7) / 8);
    k_down2<T, 8><<<g, NT, down_smem<8>(sizeof(T)), s>>>(u_in, zero_init ? 1 : 0, b, qt<T>(F), dt<T>(F), c, F.m,
                                                           Cl.m, u_out, bc);
  } else {
    dim3 g((Cl.m + 15) / 16, (Cl.m + 15) / 16);
    k_down2<T, 16><<<g, NT, down_smem<16>(sizeof(T)), s>>>(u_in, zero_init ? 1 : 0, b, qt<T>(F), dt<T>(F), c,
                                                             F.m, Cl.m, u_out, bc);
  }
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_up2(const Level& F, const Level& Cl, const cx<T>* u_in, const cx<T>* ec, const cx<T>* b,
                       cx<T>* u_out, cudaStream_t s) {
  cx<T> c = mk<cx<T>>((T)F.c.x, (T)F.c.y);
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * (3.0 * F.N + Cl.N), 0);
  if (small_tiles(Cl.m)) {
    dim3 g((Cl.m + 7) / 8, (Cl.m + 7) / 8);
    k_up2<T, 8><<<g, NT, up_smem<8>(sizeof(T)), s>>>(u_in, ec, b, qt<T>(F), dt<T>(F), c, F.m, Cl.m, u_out);
  } else {
    dim3 g((Cl.m + 15) / 16, (Cl.m + 15) / 16);
    k_up2<T, 16><<<g, NT, up_smem<16>(sizeof(T)), s>>>(u_in, ec, b, qt<T>(F), dt<T>(F), c, F.m, Cl.m, u_out);
  }
  count_launch();
  return cudaGetLastError();
}

size_t coarse_levels_smem(int dim, const std::vector<Level>& lv, int lc, int real_bytes) {
  size_t n = 0;
  for (size_t l = lc; l < lv.size(); ++l) n += 5 * (size_t)lv[l].N;
  return n * 2 * real_bytes;
}

template <typename T>
cudaError_t launch_coarse_levels(int dim, const std::vector<Level>& lv, int lc, const double2* inv, const cx<T>* b,
                                 cx<T>* u, cudaStream_t s) {
  CoarseLevels L{};
  L.nl = (int)lv.size() - lc;
  if (L.nl > 8 || L.nl < 1) return cudaErrorInvalidValue;
  for (int i = 0; i < L.nl; ++i) {
    const Level& v = lv[lc + i];
    L.m[i] = v.m;
    L.q[i] = qt<T>(v);
    L.dinv[i] = dt<T>(v);
    L.c[i] = v.c;
  }
  size_t sm = coarse_levels_smem(dim, lv, lc, sizeof(T));
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * 2.0 * lv[lc].N, 0);
  if (dim == 2) k_coarse_levels<T, 2><<<1, 1024, sm, s>>>(L, b, u, inv);
  else k_coarse_levels<T, 3><<<1, 1024, sm, s>>>(L, b, u, inv);
  count_launch();
  return cudaGetLastError();
}

// Opt the fused kernels into the dynamic shared memory they need (done at plan
// creation on the plan's device; the coarse-level kernel gets the plan's size
// or the largest size set so far, whichever is larger).
cudaError_t prepare_fused(int dim, const std::vector<Level>& lv, int lc) {
  const int kMax = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_down2<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)down_smem<16>(4))) ||
      (e = cudaFuncSetAttribute(k_down2<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)down_smem<16>(8))) ||
      (e = cudaFuncSetAttribute(k_up2<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)up_smem<16>(4))) ||
      (e = cudaFuncSetAttribute(k_up2<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)up_smem<16>(8))) ||
      (e = cudaFuncSetAttribute(k_down2<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)down_smem<8>(8))) ||
      (e = cudaFuncSetAttribute(k_up2<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)up_smem<8>(8))))
    return e;
  size_t s8 = coarse_levels_smem(dim, lv, lc, 8);
  if (s8 > (size_t)kMax) return cudaErrorInvalidValue;
  if (dim == 2) {
    if ((e = cudaFuncSetAttribute(k_coarse_levels<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)) ||
        (e = cudaFuncSetAttribute(k_coarse_levels<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)))
      return e;
  } else {
    if ((e = cudaFuncSetAttribute(k_coarse_levels<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)) ||
        (e = cudaFuncSetAttribute(k_coarse_levels<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)))
      return e;
  }
  return cudaSuccess;
}

#define CSFF_FUSED_INST(T)                                                                                 \
  template cudaError_t launch_down2<T>(const Level&, const Level&, const cx<T>*, bool, const cx<T>*, cx<T>*, \
                                       cx<T>*, cudaStream_t);                                              \
  template cudaError_t launch_up2<T>(const Level&, const Level&, const cx<T>*, const cx<T>*, const cx<T>*,   \
                                     cx<T>*, cudaStream_t);                                                \
  template cudaError_t launch_coarse_levels<T>(int, const std::vector<Level>&, int, const double2*,         \
                                               const cx<T>*, cx<T>*, cudaStream_t);
CSFF_FUSED_INST(double)
CSFF_FUSED_INST(float)

}  // namespace csff
