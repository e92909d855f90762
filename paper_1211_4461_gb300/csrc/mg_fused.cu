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
// up(l) reads it and writes the final iterate back.  Since a red update never
// reads the red point's own old value, both kernels read only the black
// points of the incoming iterate, and down(l) writes only those.  The tile
// bodies live in mg_tiles.cuh (shared with the persistent batched kernel).
#include "mg_tiles.cuh"

namespace csff {
namespace {

using tiles::Geo;
using tiles::NT;
using tiles::CoarseLevels;

// FP64 16-point tiles need 75 KB of shared memory (three CTAs per SM)
template <typename T, int TC> constexpr int tile_min_ctas() { return (sizeof(T) == 8 && TC == 16) ? 3 : 8; }

template <typename T, int TC, bool G1>
__global__ void __launch_bounds__(NT, tile_min_ctas<T, TC>()) k_down2(const cx<T>* __restrict__ u_in, int zero_init,
                                              const cx<T>* __restrict__ b, const tiles::LevelCoef<T> K, cx<T> c,
                                              int m, int mc, cx<T>* __restrict__ u_out, cx<T>* __restrict__ bc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_prologue();
  tiles::down_tile<T, TC, false, G1>(blockIdx.x * TC, blockIdx.y * TC, u_in, zero_init, b, K, c, m, mc, u_out, bc,
                                 smem_raw);
}

template <typename T, int TC, bool G1>
__global__ void __launch_bounds__(NT, tile_min_ctas<T, TC>()) k_up2(const cx<T>* __restrict__ u_in, const cx<T>* __restrict__ ec,
                                            const cx<T>* __restrict__ b, const tiles::LevelCoef<T> K, cx<T> c,
                                            int m, int mc, cx<T>* __restrict__ u_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the tile waits for its predecessor itself, after its window copies
  tiles::up_tile<T, TC, false, G1>(blockIdx.x * TC, blockIdx.y * TC, u_in, ec, b, K, c, m, mc, u_out, smem_raw);
}

template <typename T, int D, typename TI = T>
__global__ void __launch_bounds__(1024) k_coarse_levels(CoarseLevels L, const cx<T>* __restrict__ b_top,
                                                        cx<T>* __restrict__ u_top, const cx<TI>* __restrict__ inv) {
  extern __shared__ unsigned char smem_raw[];
  pdl_prologue();
  tiles::coarse_levels_block<T, D, false, TI>(L, b_top, u_top, inv, smem_raw);
}

template <typename T> const cx<T>* qt(const Level& L);
template <> const double2* qt<double>(const Level& L) { return L.q64; }
template <> const float2* qt<float>(const Level& L) { return L.q32; }
template <typename T> const cx<T>* dt(const Level& L);
template <> const double2* dt<double>(const Level& L) { return L.dinv64; }
template <> const float2* dt<float>(const Level& L) { return L.dinv32; }

// the tiles' view of a level's coefficients (formed from factors in FP32)
template <typename T> tiles::LevelCoef<T> level_coef(const Level& L);
template <> tiles::LevelCoef<double> level_coef<double>(const Level& L) {
  tiles::LevelCoef<double> K;
  K.q = L.q64;
  K.dinv = L.dinv64;
  return K;
}
template <> tiles::LevelCoef<float> level_coef<float>(const Level& L) {
  tiles::LevelCoef<float> K;
  K.fac = L.fac32;
  K.ng = L.ng;
  K.k2 = (float)L.k2;
  return K;
}
template <typename T> int coef_ng(const Level& L) { return tiles::formed_coef<T>() ? L.ng : 0; }

}  // namespace

template <int TC> size_t down_smem(int rb, int ng) { return tiles::down_smem_elems<TC>(ng, rb == 8) * 2 * rb; }
template <int TC> size_t up_smem(int rb, int ng) { return tiles::up_smem_elems<TC>(ng, rb == 8) * 2 * rb; }
// tiles of 16 coarse points on levels with at least 128 of them (the 513^2
// level too: its 256 tiles of 16 do less halo work than 1024 tiles of 8 and
// leave most of the GPU to the other maps of a concurrent step, 2-3 % faster
// there; one map alone ran 3-5 % slower that way), tiles of 8 below
static bool small_tiles(int mc) { return ((mc + 15) / 16) * ((mc + 15) / 16) < 128; }

// the down and up kernels for a tile size, specialised for a single Gaussian
// in FP32 (its x factors then stay in registers)
template <typename T, int TC>
cudaError_t down2_tc(dim3 g, size_t smem, bool g1, cudaStream_t s, const cx<T>* u_in, int zi, const cx<T>* b,
                     const tiles::LevelCoef<T>& K, cx<T> c, int m, int mc, cx<T>* u_out, cx<T>* bc) {
  if constexpr (tiles::formed_coef<T>())
    if (g1) return launch_pdl(k_down2<T, TC, true>, g, dim3(NT), smem, s, u_in, zi, b, K, c, m, mc, u_out, bc);
  return launch_pdl(k_down2<T, TC, false>, g, dim3(NT), smem, s, u_in, zi, b, K, c, m, mc, u_out, bc);
}
template <typename T, int TC>
cudaError_t up2_tc(dim3 g, size_t smem, bool g1, cudaStream_t s, const cx<T>* u_in, const cx<T>* ec,
                   const cx<T>* b, const tiles::LevelCoef<T>& K, cx<T> c, int m, int mc, cx<T>* u_out) {
  if constexpr (tiles::formed_coef<T>())
    if (g1) return launch_pdl(k_up2<T, TC, true>, g, dim3(NT), smem, s, u_in, ec, b, K, c, m, mc, u_out);
  return launch_pdl(k_up2<T, TC, false>, g, dim3(NT), smem, s, u_in, ec, b, K, c, m, mc, u_out);
}

template <typename T>
cudaError_t launch_down2(const Level& F, const Level& Cl, const cx<T>* u_in, bool zero_init, const cx<T>* b,
                         cx<T>* u_out, cx<T>* bc, cudaStream_t s, bool finest) {
  cx<T> c = mk<cx<T>>((T)F.c.x, (T)F.c.y);
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * (3.0 * F.N + Cl.N), 0,
               sizeof(T) == 4 ? PF_TILES32 : -1, sizeof(T) == 4 && finest ? PF_TILES32_FINE : -1);
  const tiles::LevelCoef<T> K = level_coef<T>(F);
  const int ng = coef_ng<T>(F);
  cudaError_t e;
  if (small_tiles(Cl.m)) {
    dim3 g((Cl.m + 7) / 8, (Cl.m + 7) / 8);
    e = down2_tc<T, 8>(g, down_smem<8>(sizeof(T), ng), ng == 1, s, u_in, zero_init ? 1 : 0, b, K, c, F.m, Cl.m,
                       u_out, bc);
  } else {
    dim3 g((Cl.m + 15) / 16, (Cl.m + 15) / 16);
    e = down2_tc<T, 16>(g, down_smem<16>(sizeof(T), ng), ng == 1, s, u_in, zero_init ? 1 : 0, b, K, c, F.m,
                        Cl.m, u_out, bc);
  }
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_up2(const Level& F, const Level& Cl, const cx<T>* u_in, const cx<T>* ec, const cx<T>* b,
                       cx<T>* u_out, cudaStream_t s, bool finest) {
  cx<T> c = mk<cx<T>>((T)F.c.x, (T)F.c.y);
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * (3.0 * F.N + Cl.N), 0,
               sizeof(T) == 4 ? PF_TILES32 : -1, sizeof(T) == 4 && finest ? PF_TILES32_FINE : -1);
  const tiles::LevelCoef<T> K = level_coef<T>(F);
  const int ng = coef_ng<T>(F);
  cudaError_t e;
  if (small_tiles(Cl.m)) {
    dim3 g((Cl.m + 7) / 8, (Cl.m + 7) / 8);
    e = up2_tc<T, 8>(g, up_smem<8>(sizeof(T), ng), ng == 1, s, u_in, ec, b, K, c, F.m, Cl.m, u_out);
  } else {
    dim3 g((Cl.m + 15) / 16, (Cl.m + 15) / 16);
    e = up2_tc<T, 16>(g, up_smem<16>(sizeof(T), ng), ng == 1, s, u_in, ec, b, K, c, F.m, Cl.m, u_out);
  }
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

size_t coarse_levels_smem(int dim, const std::vector<Level>& lv, int lc, int real_bytes) {
  return tiles::coarse_levels_elems(lv, lc) * 2 * real_bytes;
}

template <typename T>
cudaError_t launch_coarse_levels(int dim, const std::vector<Level>& lv, int lc, const cx<T>* inv,
                                 const double2* inv64, const cx<T>* b, cx<T>* u, cudaStream_t s) {
  CoarseLevels L{};
  L.nl = (int)lv.size() - lc;
  if (L.nl > 8 || L.nl < 1) return cudaErrorInvalidValue;
  for (int i = 0; i < L.nl; ++i) {
    const Level& v = lv[lc + i];
    L.m[i] = v.m;
    L.q[i] = qt<T>(v);
    L.dinv[i] = dt<T>(v);
    L.c[i] = v.c;
    L.c32[i] = make_float2((float)v.c.x, (float)v.c.y);
  }
  size_t sm = coarse_levels_smem(dim, lv, lc, sizeof(T));
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * 2.0 * lv[lc].N, 0);
  cudaError_t e;
  if (sizeof(T) == 4 && inv64)
    e = (dim == 2) ? launch_pdl(k_coarse_levels<T, 2, double>, dim3(1), dim3(1024), sm, s, L, b, u, inv64)
                   : launch_pdl(k_coarse_levels<T, 3, double>, dim3(1), dim3(1024), sm, s, L, b, u, inv64);
  else
    e = (dim == 2) ? launch_pdl(k_coarse_levels<T, 2>, dim3(1), dim3(1024), sm, s, L, b, u, inv)
                   : launch_pdl(k_coarse_levels<T, 3>, dim3(1), dim3(1024), sm, s, L, b, u, inv);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Opt the fused kernels into the dynamic shared memory they need (done at plan
// creation on the plan's device; the coarse-level kernel gets the plan's size
// or the largest size set so far, whichever is larger).
cudaError_t prepare_fused(int dim, const std::vector<Level>& lv, int lc) {
  const int kMax = 227 * 1024;
  cudaError_t e;
  // the tiles stay below the default 48 KB (FP64: no factor windows; FP32:
  // at most 8 Gaussians)
  if ((e = cudaFuncSetAttribute(k_down2<double, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)down_smem<16>(8, 0))) ||
      (e = cudaFuncSetAttribute(k_up2<double, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)up_smem<16>(8, 0))))
    return e;
  static_assert(tiles::down_smem_elems<16>(8, false) * 8 <= 48 * 1024 &&
                    tiles::up_smem_elems<16>(8, false) * 8 <= 48 * 1024 &&
                    tiles::down_smem_elems<8>(0, true) * 16 <= 48 * 1024 &&
                    tiles::up_smem_elems<8>(0, true) * 16 <= 48 * 1024,
                "fused tile shared memory");
  size_t s8 = coarse_levels_smem(dim, lv, lc, 8);
  if (s8 > (size_t)kMax) return cudaErrorInvalidValue;
  if (dim == 2) {
    if ((e = cudaFuncSetAttribute(k_coarse_levels<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)) ||
        (e = cudaFuncSetAttribute(k_coarse_levels<float, 2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMax)) ||
        (e = cudaFuncSetAttribute(k_coarse_levels<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)))
      return e;
  } else {
    if ((e = cudaFuncSetAttribute(k_coarse_levels<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)) ||
        (e = cudaFuncSetAttribute(k_coarse_levels<float, 3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMax)) ||
        (e = cudaFuncSetAttribute(k_coarse_levels<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax)))
      return e;
  }
  return cudaSuccess;
}

#define CSFF_FUSED_INST(T)                                                                                 \
  template cudaError_t launch_down2<T>(const Level&, const Level&, const cx<T>*, bool, const cx<T>*, cx<T>*, \
                                       cx<T>*, cudaStream_t, bool);                                        \
  template cudaError_t launch_up2<T>(const Level&, const Level&, const cx<T>*, const cx<T>*, const cx<T>*,   \
                                     cx<T>*, cudaStream_t, bool);                                          \
  template cudaError_t launch_coarse_levels<T>(int, const std::vector<Level>&, int, const cx<T>*,           \
                                               const double2*, const cx<T>*, cx<T>*, cudaStream_t);
CSFF_FUSED_INST(double)
CSFF_FUSED_INST(float)

}  // namespace csff
