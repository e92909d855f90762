// The learned smoother's network (bias-free 3x3 convolutions 2 -> 16 -> 16 -> 2,
// ReLU between layers, BF16 weights and activations, FP32 accumulation) for
// inference, its three layers fused per output tile in shared memory on the
// tensor cores.  run_tile (tcgen05, tensor memory) serves the stand-alone
// inference kernel; mmat::run_tile (warp-level mma.sync) the batched
// persistent solve.
//
// An output tile of TW x TH pixels needs layer-2 activations on a one-pixel
// ring around it, layer-1 activations on a two-pixel ring and the input on a
// three-pixel ring: a region of RW x RH = (TW + 6) x (TH + 6) pixels, its
// pixels numbered row-major (region row p = y RW + x).  Layer L is computed on
// the run of region rows from (L, L) to (RW-1-L, RH-1-L), in blocks of 128
// consecutive rows, as tcgen05 GEMMs M128 N16 K16 (BF16 operands, FP32
// accumulators in tensor memory):
//   layer 1: the input entry E[p] = (x(p-1), x(p), x(p+1)) of both channels
//     (six values and two zeros: one 16-byte K group) is one filter row of
//     the 3x3 stencil, so two MMAs cover it, with the K groups (E[p-RW], E[p])
//     and (E[p+RW], E[p+2RW]) (the last with zero weights);
//   layers 2 and 3: nine MMAs, one per tap (a, b), each reading the
//     activation planes shifted by (a-1) RW + (b-1) rows.
// A shift by whole rows is a start-address offset: activations are kept as
// two planes (channels 0-7 and 8-15) of 16-byte rows, the no-swizzle K-major
// operand layout (8-row core matrices 128 bytes apart, the two K groups one
// plane apart).  Pixels outside the patch are zero in every layer (zero
// padding per layer, as in the layer-by-layer kernels).  A row whose
// neighbourhood leaves the region at its depth holds a value that only rows of
// the same kind read; every row the MMAs read lies inside the planes and is
// finite (the planes are zeroed before use, the input rows past the region are
// rewritten as zeros for every tile).  Each layer's MMAs complete on an
// mbarrier (bounded wait).
//
// Weights in the flat (out, in, a, b) order of the layer-by-layer kernels:
// layer 1 (288 values), layer 2 (2304), layer 3 (288).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace csff {
namespace nettile {

constexpr int NW1 = 16 * 2 * 9, NW2 = 16 * 16 * 9;
constexpr int TW = 32, TH = 16, RW = TW + 6, RH = TH + 6, R = RW * RH;
constexpr __host__ __device__ int first_row(int L) { return L * RW + L; }
constexpr __host__ __device__ int n_rows(int L) { return (RH - 2 * L) * RW - 2 * L; }
constexpr __host__ __device__ int n_blocks(int L) { return (n_rows(L) + 127) / 128; }
constexpr int PR = 896;                          // rows per plane
constexpr int PLANE = PR * 16;
// h1 in planes 0-1, h2 in planes 2-3; plane 2 holds the input entries until
// layer 1's MMAs have completed, plane 3 the staged input until layer 2's
// epilogue
constexpr int OFF_H1 = 0, OFF_H2 = 2 * PLANE, OFF_E = OFF_H2, OFF_STAGE = 3 * PLANE;
constexpr int PLANES_BYTES = 4 * PLANE;
constexpr int SW = RW + 2, SR = SW * RH;         // staged input: the region widened by a column on each side
// weight operands (20 of 16 x 16: layer 1 two, layers 2 and 3 nine each), then
// the mbarrier and the tensor-memory address slot
constexpr int W_OPS = 20 * 512;
constexpr int WREG_BYTES = W_OPS + 64;
constexpr int NT = 256;
constexpr int SPT = (SR + NT - 1) / NT;          // staged input values per thread
constexpr int TMEM_COLS = 128;
constexpr long long WAIT_LIMIT = 1ll << 26;
static_assert(R <= PR, "region rows");
static_assert(first_row(1) - RW >= 0, "input entries read before the plane");
static_assert(first_row(1) + n_blocks(1) * 128 - 1 + 2 * RW < PR, "input entries read past the plane");
static_assert(first_row(2) - RW - 1 >= 0 && first_row(3) - RW - 1 >= 0, "activations read before the plane");
static_assert(first_row(2) + n_blocks(2) * 128 - 1 + RW + 1 < PR, "h1 read past the plane");
static_assert(first_row(3) + n_blocks(3) * 128 - 1 + RW + 1 < PR, "h2 read past the plane");
static_assert(first_row(1) + n_blocks(1) * 128 <= PR && first_row(2) + n_blocks(2) * 128 <= PR, "writes");
static_assert(n_blocks(1) * 16 <= TMEM_COLS && n_blocks(2) * 16 <= TMEM_COLS && n_blocks(3) * 16 <= TMEM_COLS,
              "tensor memory");
static_assert(SR * 8 <= PLANE, "staged input");
static_assert((n_blocks(3) + 1) / 2 <= 3, "output pixels per thread");

// one output tile: the patch (input x, output y, H x W pixels, row-major) and
// the region's origin in it (tile origin - 3)
struct Tile {
  const float2* x;
  float2* y;
  int H, W, gx0, gy0;
};

// per-CTA state: shared-memory addresses, tensor memory, mbarrier phase
struct Ctx {
  unsigned char* planes;
  uint32_t splanes, sw, bar, tmem, tl, idesc, phase;
  int half, quarter, lane;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// no-swizzle K-major descriptor: 16-byte rows, 8-row core matrices 128 bytes
// apart, K groups lbo bytes apart
__device__ __forceinline__ uint64_t ns_desc(uint32_t a, uint32_t lbo) {
  return (uint64_t)((a & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) | ((uint64_t)(128 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// two FP32 values to packed BF16 (lo in the low half), round to nearest even;
// with ReLU folded into the conversion
__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ uint32_t bf2_relu(uint32_t lo, uint32_t hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(__uint_as_float(hi)), "f"(__uint_as_float(lo)));
  return d;
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t phase) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t d;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(d)
        : "r"(bar), "r"(phase)
        : "memory");
    if (d) return true;
  }
  return false;
}

// Once per CTA, all threads: the mbarrier, TMEM_COLS columns of tensor memory
// (warp 0) and the weight operands in wreg (element (n, k) of operand t at
// (k / 8) 256 + (n / 8) 128 + (n % 8) 16 + (k % 8) 2).  The planes are not
// touched (zero_planes).
__device__ inline void setup(Ctx& c, unsigned char* planes, unsigned char* wreg, const __nv_bfloat16* __restrict__ wb) {
  const int tid = threadIdx.x, warp = tid >> 5;
  c.planes = planes;
  c.splanes = saddr(planes);
  c.sw = saddr(wreg);
  c.bar = c.sw + W_OPS;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(wreg + W_OPS + 16);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c.bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int i = tid; i < 20 * 256; i += blockDim.x) {
    const int t = i >> 8, n = (i >> 4) & 15, k = i & 15;
    __nv_bfloat16 v = zero;
    if (t < 2) {
      // layer 1, K group (k / 8) of MMA t: filter row dy, entry e = 2 (dx + 1) + channel
      const int grp = k >> 3, e = k & 7;
      const int dy = (t == 0) ? grp - 1 : grp + 1;
      if (e < 6 && dy <= 1) v = wb[(n * 2 + (e & 1)) * 9 + (dy + 1) * 3 + (e >> 1)];
    } else if (t < 11) {
      v = wb[NW1 + (n * 16 + k) * 9 + (t - 2)];
    } else if (n < 2) {
      v = wb[NW1 + NW2 + (n * 16 + k) * 9 + (t - 11)];
    }
    *reinterpret_cast<__nv_bfloat16*>(wreg + t * 512 + (k >> 3) * 256 + (n >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) =
        v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  c.tmem = *tslot;
  c.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  c.quarter = warp & 3;                           // tensor-memory lanes 32 quarter ..
  c.half = warp >> 2;                             // blocks of this parity
  c.lane = tid & 31;
  c.tl = c.tmem + ((uint32_t)(32 * c.quarter) << 16);
  c.phase = 0;
}

// all threads; the planes' previous users must be done (barrier before)
__device__ inline void zero_planes(const Ctx& c) {
  for (int i = threadIdx.x; i < PLANES_BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(c.planes)[i] = make_uint4(0, 0, 0, 0);
}

// all threads, after the last tile: frees the tensor memory
__device__ inline void teardown(const Ctx& c) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "n"(TMEM_COLS));
}

// the tile's staged input (x on the widened region, zero outside the patch)
__device__ __forceinline__ void load_x(const Tile& T, float2 (&xr)[SPT]) {
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    const int i = threadIdx.x + k * NT;
    const int sy = i / SW, sx = i - sy * SW;
    const int gy = T.gy0 + sy, gx = T.gx0 - 1 + sx;
    xr[k] = (i < SR && gy >= 0 && gy < T.H && gx >= 0 && gx < T.W) ? T.x[(long long)gy * T.W + gx]
                                                                  : make_float2(0.f, 0.f);
  }
}

// waits for the MMAs just committed; on a timeout the CTA records it, waits
// once more (bounded) for MMAs still in flight and gives up
__device__ __forceinline__ bool layer_done(Ctx& c, int* err) {
  const bool d = wait_bar(c.bar, c.phase);
  if (!__syncthreads_and(d ? 1 : 0)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    wait_bar(c.bar, c.phase);
    return false;
  }
  c.phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

__device__ __forceinline__ void commit(const Ctx& c) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(c.bar) : "memory");
}

// generic-proxy shared-memory writes of every thread become visible to the
// tensor core
__device__ __forceinline__ void to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
}

// hidden layer's epilogue: ReLU and BF16 rounding in one conversion, zero
// outside the patch, into the two planes at byte offset off
__device__ __forceinline__ void hidden(const Ctx& c, const Tile& T, int L, int off) {
  const int nb = n_blocks(L);
  for (int j = c.half; j < nb; j += 2) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(c.tl + (uint32_t)(j * 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int p = first_row(L) + j * 128 + 32 * c.quarter + c.lane;
    const int ry = p / RW, rx = p - ry * RW;
    const int gy = T.gy0 + ry, gx = T.gx0 + rx;
    const bool in = ry < RH && gy >= 0 && gy < T.H && gx >= 0 && gx < T.W;
    uint4 lo = make_uint4(0, 0, 0, 0), hi = make_uint4(0, 0, 0, 0);
    if (in) {
      lo = make_uint4(bf2_relu(v[0], v[1]), bf2_relu(v[2], v[3]), bf2_relu(v[4], v[5]), bf2_relu(v[6], v[7]));
      hi = make_uint4(bf2_relu(v[8], v[9]), bf2_relu(v[10], v[11]), bf2_relu(v[12], v[13]), bf2_relu(v[14], v[15]));
    }
    *reinterpret_cast<uint4*>(c.planes + off + p * 16) = lo;
    *reinterpret_cast<uint4*>(c.planes + off + PLANE + p * 16) = hi;
  }
}

// nine taps from the planes at in_off with weight operands from b_op on: the A
// descriptor of tap (a, b) is the block's by (a-1) RW + (b-1) rows (one unit
// of the 16-byte address field per row); one thread
__device__ __forceinline__ void taps(const Ctx& c, int L, int in_off, int b_op) {
  const uint64_t bd0 = ns_desc(c.sw + b_op * 512, 256);
  for (int j = 0; j < n_blocks(L); ++j) {
    const uint64_t ad0 = ns_desc(c.splanes + in_off + (first_row(L) + j * 128 - RW - 1) * 16, PLANE);
#pragma unroll
    for (int t = 0; t < 9; ++t)
      mma(c.tmem + j * 16, ad0 + (uint64_t)((t / 3) * RW + (t % 3)), bd0 + (uint64_t)(t * 32), c.idesc,
          t > 0 ? 1u : 0u);
  }
  commit(c);
}

// One tile, all threads: y = N(scale x) (accumulate: y += N(scale x)) on the
// tile's output pixels.  xr holds the tile's staged input (load_x); once it is
// staged, the next tile's input (next, if not null) is loaded into it while
// this tile's MMAs run.  Returns false after a timed-out wait (err set).
static __device__ __forceinline__ bool run_tile(Ctx& c, const Tile& T, float2 (&xr)[SPT], float scale, int accumulate,
                                               int* err, const Tile* next) {
  const int tid = threadIdx.x;
  float2* stage = reinterpret_cast<float2*>(c.planes + OFF_STAGE);
#pragma unroll
  for (int k = 0; k < SPT; ++k)
    if (tid + k * NT < SR) stage[tid + k * NT] = xr[k];
  __syncthreads();
  // input entries (zero past the region)
  for (int p = tid; p < PR; p += NT) {
    uint4 ev = make_uint4(0, 0, 0, 0);
    if (p < R) {
      const int ry = p / RW, rx = p - ry * RW;
      const float2* sp = stage + ry * SW + rx;       // x(p - 1), x(p), x(p + 1)
      ev.x = bf2(sp[0].x * scale, sp[0].y * scale);
      ev.y = bf2(sp[1].x * scale, sp[1].y * scale);
      ev.z = bf2(sp[2].x * scale, sp[2].y * scale);
    }
    *reinterpret_cast<uint4*>(c.planes + OFF_E + p * 16) = ev;
  }
  // this thread's output pixels, and the next tile's input
  float2 yv[3];
  if (accumulate) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int j = c.half + 2 * i;
      const int p = first_row(3) + j * 128 + 32 * c.quarter + c.lane;
      const int ry = p / RW, rx = p - ry * RW;
      const int gy = T.gy0 + ry, gx = T.gx0 + rx;
      yv[i] = (j < n_blocks(3) && rx >= 3 && rx < RW - 3 && ry >= 3 && ry < RH - 3 && gx < T.W && gy < T.H)
                  ? T.y[(long long)gy * T.W + gx]
                  : make_float2(0.f, 0.f);
    }
  }
  if (next) load_x(*next, xr);
  to_async();
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint64_t bd = ns_desc(c.sw, 256);
    for (int j = 0; j < n_blocks(1); ++j) {
      const uint64_t ad = ns_desc(c.splanes + OFF_E + (first_row(1) + j * 128 - RW) * 16, RW * 16);
      mma(c.tmem + j * 16, ad, bd, c.idesc, 0);
      mma(c.tmem + j * 16, ad + 2 * RW, bd + 32, c.idesc, 1);     // rows + 2 RW, weights + 512 bytes
    }
    commit(c);
  }
  if (!layer_done(c, err)) return false;
  hidden(c, T, 1, OFF_H1);
  to_async();
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    taps(c, 2, OFF_H1, 2);
  }
  if (!layer_done(c, err)) return false;
  hidden(c, T, 2, OFF_H2);
  to_async();
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    taps(c, 3, OFF_H2, 11);
  }
  if (!layer_done(c, err)) return false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = c.half + 2 * i;
    if (j >= n_blocks(3)) break;
    uint32_t v0, v1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(v0), "=r"(v1) : "r"(c.tl + (uint32_t)(j * 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int p = first_row(3) + j * 128 + 32 * c.quarter + c.lane;
    const int ry = p / RW, rx = p - ry * RW;
    const int gy = T.gy0 + ry, gx = T.gx0 + rx;
    if (rx >= 3 && rx < RW - 3 && ry >= 3 && ry < RH - 3 && gx < T.W && gy < T.H) {
      const long long idx = (long long)gy * T.W + gx;
      const float a0 = __uint_as_float(v0), a1 = __uint_as_float(v1);
      T.y[idx] = accumulate ? make_float2(yv[i].x + a0, yv[i].y + a1) : make_float2(a0, a1);
    }
  }
  // tensor memory and the planes are reused by the next tile
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

// ---- The same tile on the warp-level tensor-core instructions (mma.sync) -----
// For kernels that must not contain tensor-memory instructions: a cooperative
// launch is sized by an occupancy calculation that admits one CTA per SM for
// any kernel with them (the batched persistent kernel).  Same planes, input
// entries, regions and results as run_tile (accumulation order aside); the
// weight operands sit in shared memory as [operand][n][k] rows of 32 bytes.
// Warp w computes rows 16 w .. 16 w + 15 of every 128-row block with
// m16n8k16 BF16 MMAs: the A fragment of a tap is read by ldmatrix from the
// shifted rows of the two planes (16-byte rows, any row offset), the B
// fragment from the weight rows; accumulators stay in registers and the
// epilogues store from them.  No asynchronous proxy and no waits are involved.
namespace mmat {

__device__ __forceinline__ void ldm_x4(uint32_t addr, uint32_t (&a)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldm_x2(uint32_t addr, uint32_t (&b)[2]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(b[0]), "=r"(b[1]) : "r"(addr));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct Ctx {
  unsigned char* planes;
  uint32_t splanes, sw;
};

// all threads: the weight operands in wreg ([operand t][n][k], 512 bytes each,
// the same 20 operands as the tensor-memory path)
__device__ inline void setup(Ctx& c, unsigned char* planes, unsigned char* wreg, const __nv_bfloat16* __restrict__ wb) {
  c.planes = planes;
  c.splanes = saddr(planes);
  c.sw = saddr(wreg);
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int i = threadIdx.x; i < 20 * 256; i += blockDim.x) {
    const int t = i >> 8, n = (i >> 4) & 15, k = i & 15;
    __nv_bfloat16 v = zero;
    if (t < 2) {
      const int grp = k >> 3, e = k & 7;
      const int dy = (t == 0) ? grp - 1 : grp + 1;
      if (e < 6 && dy <= 1) v = wb[(n * 2 + (e & 1)) * 9 + (dy + 1) * 3 + (e >> 1)];
    } else if (t < 11) {
      v = wb[NW1 + (n * 16 + k) * 9 + (t - 2)];
    } else if (n < 2) {
      v = wb[NW1 + NW2 + (n * 16 + k) * 9 + (t - 11)];
    }
    *reinterpret_cast<__nv_bfloat16*>(wreg + t * 512 + n * 32 + k * 2) = v;
  }
  __syncthreads();
}

// B fragment of operand t, n-half h (lanes 0-15 give the row addresses)
__device__ __forceinline__ void load_b(const Ctx& c, int t, int h, int lane, uint32_t (&b)[2]) {
  ldm_x2(c.sw + t * 512 + (8 * h + (lane & 7)) * 32 + ((lane >> 3) & 1) * 16, b);
}

// hidden layer's epilogue from the accumulators of rows r0, r0 + 8 (n-halves h)
__device__ __forceinline__ void hidden_store(const Ctx& c, const Tile& T, int r0, int lane, const float (&acc)[2][4],
                                             int off) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int p = r0 + 8 * s;
    const int ry = p / RW, rx = p - ry * RW;
    const int gy = T.gy0 + ry, gx = T.gx0 + rx;
    const bool in = ry < RH && gy >= 0 && gy < T.H && gx >= 0 && gx < T.W;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t v = in ? bf2_relu(__float_as_uint(acc[h][2 * s]), __float_as_uint(acc[h][2 * s + 1])) : 0u;
      *reinterpret_cast<uint32_t*>(c.planes + off + h * PLANE + p * 16 + 4 * (lane & 3)) = v;
    }
  }
}

// One tile, all threads (see run_tile); returns true.
static __device__ __forceinline__ bool run_tile(const Ctx& c, const Tile& T, float2 (&xr)[SPT], float scale,
                                               int accumulate, const Tile* next) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* stage = reinterpret_cast<float2*>(c.planes + OFF_STAGE);
#pragma unroll
  for (int k = 0; k < SPT; ++k)
    if (tid + k * NT < SR) stage[tid + k * NT] = xr[k];
  __syncthreads();
  for (int p = tid; p < PR; p += NT) {
    uint4 ev = make_uint4(0, 0, 0, 0);
    if (p < R) {
      const int ry = p / RW, rx = p - ry * RW;
      const float2* sp = stage + ry * SW + rx;
      ev.x = bf2(sp[0].x * scale, sp[0].y * scale);
      ev.y = bf2(sp[1].x * scale, sp[1].y * scale);
      ev.z = bf2(sp[2].x * scale, sp[2].y * scale);
    }
    *reinterpret_cast<uint4*>(c.planes + OFF_E + p * 16) = ev;
  }
  if (next) load_x(*next, xr);
  __syncthreads();
  const int lrow = lane & 15, lk = lane >= 16 ? 1 : 0;
  // layer 1: two K16 steps, K groups (E[p - RW], E[p]) and (E[p + RW], E[p + 2 RW])
  for (int j = 0; j < n_blocks(1); ++j) {
    const int r0 = first_row(1) + j * 128 + 16 * warp;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      uint32_t a[4];
      ldm_x4(c.splanes + OFF_E + (r0 + lrow + (m == 0 ? -RW : RW) + lk * RW) * 16, a);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t b[2];
        load_b(c, m, h, lane, b);
        mma16816(acc[h], a, b);
      }
    }
    hidden_store(c, T, r0 + (lane >> 2), lane, acc, OFF_H1);
  }
  __syncthreads();
  // layer 2: nine taps from the h1 planes
  for (int j = 0; j < n_blocks(2); ++j) {
    const int r0 = first_row(2) + j * 128 + 16 * warp;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      uint32_t a[4];
      ldm_x4(c.splanes + OFF_H1 + lk * PLANE + (r0 + lrow + (t / 3 - 1) * RW + (t % 3 - 1)) * 16, a);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t b[2];
        load_b(c, 2 + t, h, lane, b);
        mma16816(acc[h], a, b);
      }
    }
    hidden_store(c, T, r0 + (lane >> 2), lane, acc, OFF_H2);
  }
  __syncthreads();
  // layer 3: nine taps from the h2 planes, outputs 0 and 1 of the first n-half
  for (int j = 0; j < n_blocks(3); ++j) {
    const int r0 = first_row(3) + j * 128 + 16 * warp;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      uint32_t a[4], b[2];
      ldm_x4(c.splanes + OFF_H2 + lk * PLANE + (r0 + lrow + (t / 3 - 1) * RW + (t % 3 - 1)) * 16, a);
      load_b(c, 11 + t, 0, lane, b);
      mma16816(acc, a, b);
    }
    if ((lane & 3) == 0) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int p = r0 + (lane >> 2) + 8 * s;
        const int ry = p / RW, rx = p - ry * RW;
        const int gy = T.gy0 + ry, gx = T.gx0 + rx;
        if (rx >= 3 && rx < RW - 3 && ry >= 3 && ry < RH - 3 && gx < T.W && gy < T.H) {
          const long long idx = (long long)gy * T.W + gx;
          const float a0 = acc[2 * s], a1 = acc[2 * s + 1];
          if (accumulate) {
            const float2 u = T.y[idx];
            T.y[idx] = make_float2(u.x + a0, u.y + a1);
          } else {
            T.y[idx] = make_float2(a0, a1);
          }
        }
      }
    }
  }
  __syncthreads();        // the planes are reused by the next tile
  return true;
}

}  // namespace mmat
}  // namespace nettile
}  // namespace csff
