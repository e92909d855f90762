// Learned smoother: a bias-free 3x3 convolutional network N (2 -> 16 -> 16 -> 2
// channels, ReLU between layers) applied as u <- u + N(r) after a red-black
// sweep on the finest levels.  Complex values are two real channels.  The
// paper has no such component; it is an addition built around the method's
// own operator: the training loss is the relative residual after the learned
// step, ||r - A N(r)||^2 / ||r||^2, with A the level's rotated-grid operator.
//
// Precision: weights and activations are stored in BF16, every convolution
// accumulates in FP32, the master weights and the Adam moments are FP32.
//
// Layout: patches [B][H][W]; the residual and the output are complex FP32
// (float2); hidden activations are channels-last BF16 [B][H][W][16].
// Convolution: out[o, i, j] = sum_c sum_{a,b} w[o][c][a][b] x[c][i+a-1][j+b-1],
// zero outside the patch.  Weights are stored flat in (out, in, a, b) order,
// layer 1 then 2 then 3 (288 + 2304 + 288 values).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "csff_internal.h"
#include "net_tile.cuh"

namespace csff {
namespace {

constexpr int NP1 = 16 * 2 * 9, NP2 = 16 * 16 * 9, NP3 = 2 * 16 * 9;
constexpr int NPARAM = NP1 + NP2 + NP3;
constexpr int NTH = 256;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16(x)); }

struct Geom {
  int B, H, W;
  __host__ __device__ __forceinline__ long long npix() const { return (long long)B * H * W; }
};

// row and column of pixel p inside its patch (32-bit: the API keeps B H W
// below 2^31)
struct Pix { int i, j; };
__device__ __forceinline__ Pix pix_of(const Geom& g, long long p) {
  const int q = (int)p;
  const int t = q / g.W;
  return Pix{t % g.H, q - t * g.W};
}

// neighbour (i + a - 1, j + b - 1) of pixel p (at c) inside its patch, or -1
__device__ __forceinline__ long long nbr_at(const Geom& g, Pix c, long long p, int a, int b) {
  const int ii = c.i + a - 1, jj = c.j + b - 1;
  if (ii < 0 || ii >= g.H || jj < 0 || jj >= g.W) return -1;
  return p + (long long)(a - 1) * g.W + (b - 1);
}
__device__ __forceinline__ long long nbr(const Geom& g, long long p, int a, int b) {
  return nbr_at(g, pix_of(g, p), p, a, b);
}

// layer 1: x0 = bf16(r) (2 channels) -> h1 = bf16(relu(conv)) (16 channels).
// The weights sit in shared memory as [tap][in][out] so that the 16 output
// weights of one (tap, input channel) are four 16-byte broadcast loads for 16
// fused multiply-adds.
__global__ void k_conv1(Geom g, const float2* __restrict__ r, const __nv_bfloat16* __restrict__ w1,
                        __nv_bfloat16* __restrict__ h1) {
  __shared__ __align__(16) float ws[9][2][16];
  for (int i = threadIdx.x; i < NP1; i += blockDim.x) {
    const int o = i / 18, c = (i / 9) % 2, t = i % 9;      // w1 index (o * 2 + c) * 9 + t
    ws[t][c][o] = __bfloat162float(w1[i]);
  }
  __syncthreads();
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  float acc[16];
#pragma unroll
  for (int o = 0; o < 16; ++o) acc[o] = 0.f;
  const Pix pc = pix_of(g, p);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      long long q = nbr_at(g, pc, p, a, b);
      if (q < 0) continue;
      const float2 v = r[q];
      const float x[2] = {bf(v.x), bf(v.y)};
#pragma unroll
      for (int c = 1; c >= 0; --c) {          // channel 1 first: the order of the per-output chains
        const float4* wv = reinterpret_cast<const float4*>(&ws[a * 3 + b][c][0]);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 w = wv[q4];
          acc[4 * q4 + 0] = fmaf(w.x, x[c], acc[4 * q4 + 0]);
          acc[4 * q4 + 1] = fmaf(w.y, x[c], acc[4 * q4 + 1]);
          acc[4 * q4 + 2] = fmaf(w.z, x[c], acc[4 * q4 + 2]);
          acc[4 * q4 + 3] = fmaf(w.w, x[c], acc[4 * q4 + 3]);
        }
      }
    }
  __align__(16) __nv_bfloat16 hv[16];
#pragma unroll
  for (int o = 0; o < 16; ++o) hv[o] = __float2bfloat16(fmaxf(acc[o], 0.f));
  uint4* dst = reinterpret_cast<uint4*>(h1 + p * 16);          // 32 bytes per pixel, two vector stores
  dst[0] = *reinterpret_cast<const uint4*>(hv);
  dst[1] = *reinterpret_cast<const uint4*>(hv + 8);
}

// Layers 2 and 3 on the tensor cores (implicit GEMM): for 128 consecutive pixels
//   D[p][o] = sum_{t = 3a + b} sum_c h[nbr(p, a, b)][c] w[o][c][a][b],
// a GEMM D[128 x 16] = A[128 x 144] B[16 x 144]^T with k = 16 t + c.  A is
// gathered into shared memory (one 16-channel, 32-byte vector per pixel and
// tap; zero outside the patch) in the 128-byte-swizzled K-major layout (taps
// 0-3, 4-7 and 8 in three 64-wide chunks); B holds the weights in the same
// layout (layer 3: rows 0-1, the rest zero).  Nine tcgen05.mma (kind::f16,
// BF16 in, FP32 accumulator in tensor memory, M = 128, N = 16, K = 16 each),
// one per tap.  Epilogue: layer 2 ReLU and BF16 rounding as the CUDA-core
// layers; layer 3 the two output channels into y (stored or added).
// Persistent: a CTA builds B and allocates tensor memory once and walks the
// pixel tiles; each tile's MMAs complete on an mbarrier (bounded wait).
namespace ctc {
constexpr int TM = 128;
constexpr int A_CHUNK = TM * 128;            // bytes of one 64-wide K chunk of A
constexpr int B_CHUNK = 16 * 128;            // bytes of one 64-wide K chunk of B
constexpr int SMEM = 3 * A_CHUNK + 3 * B_CHUNK + 1024 + 64;
constexpr int CTAS_PER_SM = 4;
constexpr long long WAIT_LIMIT = 1ll << 26;
}  // namespace ctc

__device__ __forceinline__ int c_sw128(int r, int c) { return (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4); }
__device__ __forceinline__ uint32_t c_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t c_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// LAYER 2: h -> out_h = bf16(relu(conv)) (16 channels); LAYER 3: h -> y (2
// channels, FP32; accumulate: y += conv)
template <int LAYER>
__global__ void __launch_bounds__(128) k_conv_tc(Geom g, const __nv_bfloat16* __restrict__ h,
                                                 const __nv_bfloat16* __restrict__ w,
                                                 __nv_bfloat16* __restrict__ out_h, float2* __restrict__ y,
                                                 int accumulate, int* __restrict__ err) {
  constexpr int COUT = (LAYER == 2) ? 16 : 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (c_saddr(smem_raw) & 1023)) & 1023);
  unsigned char* sA = base;
  unsigned char* sB = base + 3 * ctc::A_CHUNK;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 3 * ctc::B_CHUNK);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sB + 3 * ctc::B_CHUNK + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long np = g.npix();
  const long long ntiles = (np + ctc::TM - 1) / ctc::TM;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c_saddr(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(c_saddr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // B: row o, k = 16 t + c  <-  w[(o 16 + c) 9 + t]; 8 values per 16-byte chunk
  for (int q = tid; q < 16 * 24; q += blockDim.x) {
    const int o = q / 24, kc = q % 24;          // kc: 16-byte chunk along k (18..23 padding)
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e, t = k >> 4, c = k & 15;
      v[e] = (t < 9 && o < COUT) ? w[(o * 16 + c) * 9 + t] : __float2bfloat16(0.f);
    }
    *reinterpret_cast<uint4*>(sB + (kc >> 3) * ctc::B_CHUNK + c_sw128(o, kc & 7)) =
        *reinterpret_cast<const uint4*>(v);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) |
                         ((uint32_t)(ctc::TM >> 4) << 24);
  // A rows are gathered into registers one tile ahead: the loads of tile n+1
  // are in flight while the tensor core and the epilogue work on tile n
  uint4 xa[9][2];
  auto gather = [&](long long tile) {
    const long long p = tile * ctc::TM + tid;
    const bool pv = tile < ntiles && p < np;
    const Pix pc = pv ? pix_of(g, p) : Pix{0, 0};
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const long long nq = pv ? nbr_at(g, pc, p, t / 3, t % 3) : -1;
      if (nq >= 0) {
        const uint4* src = reinterpret_cast<const uint4*>(h + nq * 16);
        xa[t][0] = src[0];
        xa[t][1] = src[1];
      } else {
        xa[t][0] = make_uint4(0, 0, 0, 0);
        xa[t][1] = make_uint4(0, 0, 0, 0);
      }
    }
  };
  gather(blockIdx.x);
  uint32_t phase = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, phase ^= 1u) {
    const long long p0 = tile * ctc::TM;
    // A: this thread's pixel row, all nine taps (32 bytes each)
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      unsigned char* dst = sA + (t >> 2) * ctc::A_CHUNK;
      const int c0 = (t & 3) * 2;
      *reinterpret_cast<uint4*>(dst + c_sw128(tid, c0)) = xa[t][0];
      *reinterpret_cast<uint4*>(dst + c_sw128(tid, c0 + 1)) = xa[t][1];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const uint64_t ad = c_desc(c_saddr(sA + (t >> 2) * ctc::A_CHUNK) + 32 * (t & 3));
        const uint64_t bd = c_desc(c_saddr(sB + (t >> 2) * ctc::B_CHUNK) + 32 * (t & 3));
        const uint32_t acc = t > 0 ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred q;\nsetp.ne.b32 q, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       c_saddr(mbar))
                   : "memory");
    }
    gather(tile + gridDim.x);
    bool done = false;
    for (long long it = 0; it < ctc::WAIT_LIMIT && !done; ++it) {
      uint32_t d;
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(d)
          : "r"(c_saddr(mbar)), "r"(phase)
          : "memory");
      done = d != 0;
    }
    // one decision for the whole CTA (every thread polls the same barrier)
    if (!__syncthreads_and(done ? 1 : 0)) {
      if (tid == 0) atomicExch(err, 1);
      // the MMAs may still be in flight: wait once more (bounded) before the
      // tensor memory is freed
      for (long long it = 0; it < ctc::WAIT_LIMIT; ++it) {
        uint32_t d;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(d)
            : "r"(c_saddr(mbar)), "r"(phase)
            : "memory");
        if (d) break;
      }
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
      const long long p = p0 + 32 * warp + lane;
      if constexpr (LAYER == 2) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((uint32_t)(32 * warp) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (p < np) {
          __align__(16) __nv_bfloat16 o[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(fmaxf(__uint_as_float(v[j]), 0.f));
          uint4* dst = reinterpret_cast<uint4*>(out_h + p * 16);
          dst[0] = *reinterpret_cast<const uint4*>(o);
          dst[1] = *reinterpret_cast<const uint4*>(o + 8);
        }
      } else {
        uint32_t v[2];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                     : "=r"(v[0]), "=r"(v[1])
                     : "r"(tmem + ((uint32_t)(32 * warp) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (p < np) {
          const float a0 = __uint_as_float(v[0]), a1 = __uint_as_float(v[1]);
          if (accumulate) {
            const float2 u = y[p];
            y[p] = make_float2(u.x + a0, u.y + a1);
          } else {
            y[p] = make_float2(a0, a1);
          }
        }
      }
    }
    // every thread is done with shared memory and tensor memory before the
    // next tile is gathered and its MMAs overwrite the accumulator
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// ---- loss: E = mask (r - A y); per-patch sums |E|^2 and |r|^2 over the mask
__device__ __forceinline__ bool in_mask(const Geom& g, long long p, int margin) {
  int j = (int)(p % g.W);
  int i = (int)((p / g.W) % g.H);
  return i >= margin && i < g.H - margin && j >= margin && j < g.W - margin;
}

__device__ __forceinline__ float2 apply_A_patch(const Geom& g, const float2* v, long long p, float2 q, float2 c,
                                                bool conj_in) {
  auto ld = [&](long long k) {
    float2 x = v[k];
    return conj_in ? make_float2(x.x, -x.y) : x;
  };
  float2 s = make_float2(0.f, 0.f);
  for (int t = 0; t < 4; ++t) {
    int a = (t == 0) ? 0 : (t == 1) ? 2 : 1;
    int b = (t == 2) ? 0 : (t == 3) ? 2 : 1;
    long long k = nbr(g, p, a, b);
    if (k >= 0) s = cadd(s, ld(k));
  }
  float2 vj = ld(p);
  float2 t = csub(cscale(vj, 4.f), s);
  return csub(cmul(c, t), cmul(q, vj));
}

__global__ void k_loss1(Geom g, const float2* __restrict__ y, const float2* __restrict__ r,
                        const float2* __restrict__ q, const float2* __restrict__ cpatch, int margin,
                        float2* __restrict__ E, double* __restrict__ sums /* [B][2]: |E|^2, |r|^2 */) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  int bpatch = (int)(p / ((long long)g.H * g.W));
  float2 e = make_float2(0.f, 0.f);
  if (in_mask(g, p, margin)) {
    float2 rv = r[p];
    e = csub(rv, apply_A_patch(g, y, p, q[p], cpatch[bpatch], false));
    atomicAdd(&sums[2 * bpatch + 0], (double)e.x * e.x + (double)e.y * e.y);
    atomicAdd(&sums[2 * bpatch + 1], (double)rv.x * rv.x + (double)rv.y * rv.y);
  }
  E[p] = e;
}

// dy = -conj(A conj(G)), G = 2 E / (S_r B)   (A is complex symmetric)
__global__ void k_loss2(Geom g, const float2* __restrict__ E, const double* __restrict__ sums,
                        const float2* __restrict__ q, const float2* __restrict__ cpatch, float2* __restrict__ G,
                        float2* __restrict__ dy, int phase) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  int bpatch = (int)(p / ((long long)g.H * g.W));
  if (phase == 0) {
    double sr = sums[2 * bpatch + 1];
    float sc = sr > 0 ? (float)(2.0 / (sr * g.B)) : 0.f;
    G[p] = cscale(E[p], sc);
  } else {
    float2 a = apply_A_patch(g, G, p, q[p], cpatch[bpatch], true);
    dy[p] = make_float2(-a.x, a.y);     // -conj(a)
  }
}

// input gradient of layer 3: dh2[c] = sum_o sum_ab w3[o][c][a][b] dy[o](p - (a-1, b-1)), masked by h2 > 0
__global__ void k_bwd3(Geom g, const float2* __restrict__ dy, const __nv_bfloat16* __restrict__ w3,
                       const __nv_bfloat16* __restrict__ h2, float* __restrict__ dh2) {
  __shared__ float ws[NP3];
  for (int i = threadIdx.x; i < NP3; i += blockDim.x) ws[i] = __bfloat162float(w3[i]);
  __syncthreads();
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.f;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      long long q = nbr(g, p, 2 - a, 2 - b);      // out pixel p - (a-1, b-1)
      if (q < 0) continue;
      float2 d = dy[q];
#pragma unroll
      for (int c = 0; c < 16; ++c)
        acc[c] = fmaf(ws[(0 * 16 + c) * 9 + a * 3 + b], d.x, fmaf(ws[(1 * 16 + c) * 9 + a * 3 + b], d.y, acc[c]));
    }
#pragma unroll
  for (int c = 0; c < 16; ++c) dh2[p * 16 + c] = __bfloat162float(h2[p * 16 + c]) > 0.f ? acc[c] : 0.f;
}

// input gradient of layer 2, masked by h1 > 0
__global__ void k_bwd2(Geom g, const float* __restrict__ dh2, const __nv_bfloat16* __restrict__ w2,
                       const __nv_bfloat16* __restrict__ h1, float* __restrict__ dh1) {
  __shared__ float ws[NP2];
  for (int i = threadIdx.x; i < NP2; i += blockDim.x) ws[i] = __bfloat162float(w2[i]);
  __syncthreads();
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.f;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      long long q = nbr(g, p, 2 - a, 2 - b);
      if (q < 0) continue;
      const float* d = dh2 + q * 16;
#pragma unroll
      for (int o = 0; o < 16; ++o) {
        float dv = d[o];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = fmaf(ws[(o * 16 + c) * 9 + a * 3 + b], dv, acc[c]);
      }
    }
#pragma unroll
  for (int c = 0; c < 16; ++c) dh1[p * 16 + c] = __bfloat162float(h1[p * 16 + c]) > 0.f ? acc[c] : 0.f;
}

// weight gradient: dw[o][c][a][b] += sum_p dout[p][o] in[c](p + (a-1, b-1)).
// INKIND 0: input is bf16(r) (2 channels from float2); 1: bf16 activations.
// DKIND 0: dout is float2 (2 channels); 1: float[16].
template <int CIN, int COUT, int INKIND, int DKIND>
__global__ void k_wgrad(Geom g, const void* __restrict__ in, const void* __restrict__ dout, float* __restrict__ dw) {
  constexpr int NPAR = COUT * CIN * 9;
  constexpr int TP = 128;                          // pixels per block
  __shared__ float sd[TP * COUT];
  const long long p0 = (long long)blockIdx.x * TP;
  for (int i = threadIdx.x; i < TP * COUT; i += blockDim.x) {
    long long p = p0 + i / COUT;
    int o = i % COUT;
    float v = 0.f;
    if (p < g.npix()) {
      if (DKIND == 0) {
        float2 d = reinterpret_cast<const float2*>(dout)[p];
        v = (o == 0) ? d.x : d.y;
      } else {
        v = reinterpret_cast<const float*>(dout)[p * COUT + o];
      }
    }
    sd[i] = v;
  }
  __syncthreads();
  for (int par = threadIdx.x; par < NPAR; par += blockDim.x) {
    int o = par / (CIN * 9), rem = par % (CIN * 9), c = rem / 9, ab = rem % 9, a = ab / 3, b = ab % 3;
    float acc = 0.f;
    for (int t = 0; t < TP; ++t) {
      long long p = p0 + t;
      if (p >= g.npix()) break;
      long long q = nbr(g, p, a, b);
      if (q < 0) continue;
      float x;
      if (INKIND == 0) {
        float2 v = reinterpret_cast<const float2*>(in)[q];
        x = bf(c == 0 ? v.x : v.y);
      } else {
        x = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(in)[q * CIN + c]);
      }
      acc = fmaf(sd[t * COUT + o], x, acc);
    }
    atomicAdd(&dw[par], acc);
  }
}

__global__ void k_adam(float* w, float* m, float* v, const float* gr, __nv_bfloat16* wb, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = gr[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16(wi);
}

// ---- Inference: the three layers fused per output tile (net_tile.cuh).
// Persistent CTAs walk the tiles of B patches; each loads the next tile's
// input while the current tile's MMAs run.
constexpr int NET_CTAS_PER_SM = 3;
constexpr int NET_SMEM = nettile::PLANES_BYTES + nettile::WREG_BYTES + 128;
static_assert(NET_CTAS_PER_SM * nettile::TMEM_COLS <= 512, "tensor memory per SM");

// tile t of B patches of H x W (tiles row-major within a patch)
__device__ __forceinline__ nettile::Tile net_tile_of(const Geom& g, const float2* x, float2* y, int tiles_x,
                                                     int tiles_y, long long t) {
  const int tx = (int)(t % tiles_x);
  const long long t2 = t / tiles_x;
  const long long off = (t2 / tiles_y) * g.H * g.W;
  return nettile::Tile{x + off, y + off, g.H, g.W, tx * nettile::TW - 3, (int)(t2 % tiles_y) * nettile::TH - 3};
}

// y = N(scale x) (accumulate: y += N(scale x)) over B patches of H x W
__global__ void __launch_bounds__(nettile::NT, NET_CTAS_PER_SM)
    k_net_fused(Geom g, const float2* __restrict__ x, float scale, const __nv_bfloat16* __restrict__ wb,
                float2* __restrict__ y, int accumulate, int* __restrict__ err) {
  using namespace nettile;
  extern __shared__ __align__(128) unsigned char fsm_raw[];
  unsigned char* base = fsm_raw + ((128 - (saddr(fsm_raw) & 127)) & 127);
  Ctx c;
  setup(c, base, base + PLANES_BYTES, wb);
  zero_planes(c);
  const int tiles_x = (g.W + TW - 1) / TW, tiles_y = (g.H + TH - 1) / TH;
  const long long ntiles = (long long)g.B * tiles_x * tiles_y;
  float2 xr[SPT];
  Tile cur = net_tile_of(g, x, y, tiles_x, tiles_y, blockIdx.x);
  if (blockIdx.x < ntiles) load_x(cur, xr);
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long nt = t + gridDim.x;
    const Tile next = net_tile_of(g, x, y, tiles_x, tiles_y, nt < ntiles ? nt : t);
    if (!run_tile(c, cur, xr, scale, accumulate, err, nt < ntiles ? &next : nullptr)) break;
    cur = next;
  }
  teardown(c);
}


// ---- The 3D network: 3x3x3 cross-correlations, the same channels (2 -> 16 ->
// 16 -> 2), on the CUDA cores with the 2D network's precision (BF16 weights and
// activations, FP32 accumulation).  Patches [B][Z][H][W]; weights (out, in, a,
// b, e), tap t = 9 a + 3 b + e reading x[z + a - 1][y + b - 1][x + e - 1].
constexpr int T3 = 27;
constexpr int NP31 = 16 * 2 * T3, NP32 = 16 * 16 * T3, NP33 = 2 * 16 * T3;
constexpr int NPARAM3 = NP31 + NP32 + NP33;

struct Geom3 {
  int B, Z, H, W;
  __host__ __device__ __forceinline__ long long npix() const { return (long long)B * Z * H * W; }
};
struct Vox { int z, y, x; };
// coordinates of voxel p inside its patch (32-bit: B Z H W < 2^31)
__device__ __forceinline__ Vox vox_of(const Geom3& g, long long p) {
  const int q = (int)p;
  const int t = q / g.W, x = q - t * g.W;
  const int t2 = t / g.H, y = t - t2 * g.H;
  return Vox{t2 % g.Z, y, x};
}
// neighbour (z + a - 1, y + b - 1, x + e - 1) of voxel p (at v), or -1
__device__ __forceinline__ long long nbr3(const Geom3& g, Vox v, long long p, int a, int b, int e) {
  const int zz = v.z + a - 1, yy = v.y + b - 1, xx = v.x + e - 1;
  if (zz < 0 || zz >= g.Z || yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return -1;
  return p + ((long long)(a - 1) * g.H + (b - 1)) * g.W + (e - 1);
}

__device__ __forceinline__ void unpack16(const __nv_bfloat16* src, float* x) {
  const uint4 a = reinterpret_cast<const uint4*>(src)[0], b = reinterpret_cast<const uint4*>(src)[1];
  const __nv_bfloat162* pa = reinterpret_cast<const __nv_bfloat162*>(&a);
  const __nv_bfloat162* pb = reinterpret_cast<const __nv_bfloat162*>(&b);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 fa = __bfloat1622float2(pa[i]), fb = __bfloat1622float2(pb[i]);
    x[2 * i] = fa.x;
    x[2 * i + 1] = fa.y;
    x[8 + 2 * i] = fb.x;
    x[8 + 2 * i + 1] = fb.y;
  }
}
__device__ __forceinline__ void store16_relu(__nv_bfloat16* dst, const float* acc) {
  __align__(16) __nv_bfloat16 hv[16];
#pragma unroll
  for (int o = 0; o < 16; ++o) hv[o] = __float2bfloat16(fmaxf(acc[o], 0.f));
  reinterpret_cast<uint4*>(dst)[0] = *reinterpret_cast<const uint4*>(hv);
  reinterpret_cast<uint4*>(dst)[1] = *reinterpret_cast<const uint4*>(hv + 8);
}

// layer 1: x0 = bf16(scale r) -> h1 = bf16(relu(conv)); weights in shared
// memory as [tap][in][out]
__global__ void k3_conv1(Geom3 g, const float2* __restrict__ r, float scale, const __nv_bfloat16* __restrict__ w1,
                         __nv_bfloat16* __restrict__ h1) {
  __shared__ __align__(16) float ws[T3][2][16];
  for (int i = threadIdx.x; i < NP31; i += blockDim.x) {
    const int o = i / (2 * T3), c = (i / T3) % 2, t = i % T3;
    ws[t][c][o] = __bfloat162float(w1[i]);
  }
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  const Vox v = vox_of(g, p);
  float acc[16];
#pragma unroll
  for (int o = 0; o < 16; ++o) acc[o] = 0.f;
  for (int t = 0; t < T3; ++t) {
    const long long q = nbr3(g, v, p, t / 9, (t / 3) % 3, t % 3);
    if (q < 0) continue;
    const float2 rv = r[q];
    const float x[2] = {bf(rv.x * scale), bf(rv.y * scale)};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float4* wv = reinterpret_cast<const float4*>(&ws[t][c][0]);
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 w = wv[q4];
        acc[4 * q4 + 0] = fmaf(w.x, x[c], acc[4 * q4 + 0]);
        acc[4 * q4 + 1] = fmaf(w.y, x[c], acc[4 * q4 + 1]);
        acc[4 * q4 + 2] = fmaf(w.z, x[c], acc[4 * q4 + 2]);
        acc[4 * q4 + 3] = fmaf(w.w, x[c], acc[4 * q4 + 3]);
      }
    }
  }
  store16_relu(h1 + p * 16, acc);
}

// layer 2: h1 -> h2 = bf16(relu(conv)); weights [tap][in][out] (27.6 KB)
__global__ void k3_conv2(Geom3 g, const __nv_bfloat16* __restrict__ h1, const __nv_bfloat16* __restrict__ w2,
                         __nv_bfloat16* __restrict__ h2) {
  __shared__ __align__(16) float ws[T3][16][16];
  for (int i = threadIdx.x; i < NP32; i += blockDim.x) {
    const int o = i / (16 * T3), c = (i / T3) % 16, t = i % T3;
    ws[t][c][o] = __bfloat162float(w2[i]);
  }
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  const Vox v = vox_of(g, p);
  float acc[16];
#pragma unroll
  for (int o = 0; o < 16; ++o) acc[o] = 0.f;
  for (int t = 0; t < T3; ++t) {
    const long long q = nbr3(g, v, p, t / 9, (t / 3) % 3, t % 3);
    if (q < 0) continue;
    float x[16];
    unpack16(h1 + q * 16, x);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float4* wv = reinterpret_cast<const float4*>(&ws[t][c][0]);
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 w = wv[q4];
        acc[4 * q4 + 0] = fmaf(w.x, x[c], acc[4 * q4 + 0]);
        acc[4 * q4 + 1] = fmaf(w.y, x[c], acc[4 * q4 + 1]);
        acc[4 * q4 + 2] = fmaf(w.z, x[c], acc[4 * q4 + 2]);
        acc[4 * q4 + 3] = fmaf(w.w, x[c], acc[4 * q4 + 3]);
      }
    }
  }
  store16_relu(h2 + p * 16, acc);
}

// layer 3: h2 -> y (2 channels, FP32; accumulate: y += conv); weights [tap][in][out]
__global__ void k3_conv3(Geom3 g, const __nv_bfloat16* __restrict__ h2, const __nv_bfloat16* __restrict__ w3,
                         float2* __restrict__ y, int accumulate) {
  __shared__ __align__(16) float2 ws[T3][16];
  for (int i = threadIdx.x; i < NP33; i += blockDim.x) {
    const int o = i / (16 * T3), c = (i / T3) % 16, t = i % T3;
    float* wf = reinterpret_cast<float*>(&ws[t][c]);
    wf[o] = __bfloat162float(w3[i]);
  }
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  const Vox v = vox_of(g, p);
  float a0 = 0.f, a1 = 0.f;
  for (int t = 0; t < T3; ++t) {
    const long long q = nbr3(g, v, p, t / 9, (t / 3) % 3, t % 3);
    if (q < 0) continue;
    float x[16];
    unpack16(h2 + q * 16, x);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float2 w = ws[t][c];
      a0 = fmaf(w.x, x[c], a0);
      a1 = fmaf(w.y, x[c], a1);
    }
  }
  if (accumulate) {
    const float2 u = y[p];
    y[p] = make_float2(u.x + a0, u.y + a1);
  } else {
    y[p] = make_float2(a0, a1);
  }
}

// ---- 3D loss: E = mask (r - A y) with the 7-point operator
__device__ __forceinline__ bool in_mask3(const Geom3& g, Vox v, int margin) {
  return v.z >= margin && v.z < g.Z - margin && v.y >= margin && v.y < g.H - margin && v.x >= margin &&
         v.x < g.W - margin;
}

__device__ __forceinline__ float2 apply_A3(const Geom3& g, const float2* f, long long p, float2 q, float2 c,
                                           bool conj_in) {
  const Vox v = vox_of(g, p);
  auto ld = [&](long long k) {
    const float2 x = f[k];
    return conj_in ? make_float2(x.x, -x.y) : x;
  };
  float2 sn = make_float2(0.f, 0.f);
  const int ax[6][3] = {{0, 1, 1}, {2, 1, 1}, {1, 0, 1}, {1, 2, 1}, {1, 1, 0}, {1, 1, 2}};
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    const long long k = nbr3(g, v, p, ax[n][0], ax[n][1], ax[n][2]);
    if (k >= 0) sn = cadd(sn, ld(k));
  }
  const float2 vj = ld(p);
  return csub(cmul(c, csub(cscale(vj, 6.f), sn)), cmul(q, vj));
}

__global__ void k3_loss1(Geom3 g, const float2* __restrict__ y, const float2* __restrict__ r,
                         const float2* __restrict__ q, const float2* __restrict__ cpatch, int margin,
                         float2* __restrict__ E, double* __restrict__ sums) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  const int bpatch = (int)(p / ((long long)g.Z * g.H * g.W));
  float2 e = make_float2(0.f, 0.f);
  if (in_mask3(g, vox_of(g, p), margin)) {
    const float2 rv = r[p];
    e = csub(rv, apply_A3(g, y, p, q[p], cpatch[bpatch], false));
    atomicAdd(&sums[2 * bpatch + 0], (double)e.x * e.x + (double)e.y * e.y);
    atomicAdd(&sums[2 * bpatch + 1], (double)rv.x * rv.x + (double)rv.y * rv.y);
  }
  E[p] = e;
}

// dy = -conj(A conj(G)), G = 2 E / (S_r B)
__global__ void k3_loss2(Geom3 g, const float2* __restrict__ E, const double* __restrict__ sums,
                         const float2* __restrict__ q, const float2* __restrict__ cpatch, float2* __restrict__ G,
                         float2* __restrict__ dy, int phase) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  const int bpatch = (int)(p / ((long long)g.Z * g.H * g.W));
  if (phase == 0) {
    const double sr = sums[2 * bpatch + 1];
    const float sc = sr > 0 ? (float)(2.0 / (sr * g.B)) : 0.f;
    G[p] = cscale(E[p], sc);
  } else {
    const float2 a = apply_A3(g, G, p, q[p], cpatch[bpatch], true);
    dy[p] = make_float2(-a.x, a.y);
  }
}

// input gradients: dh2[c] = sum_o sum_t w3[o][c][t] dy[o](p - (t - 1)) masked by
// h2 > 0; dh1 likewise from dh2 and w2, masked by h1 > 0
__global__ void k3_bwd3(Geom3 g, const float2* __restrict__ dy, const __nv_bfloat16* __restrict__ w3,
                        const __nv_bfloat16* __restrict__ h2, float* __restrict__ dh2) {
  __shared__ float ws[NP33];
  for (int i = threadIdx.x; i < NP33; i += blockDim.x) ws[i] = __bfloat162float(w3[i]);
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  const Vox v = vox_of(g, p);
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.f;
  for (int t = 0; t < T3; ++t) {
    const long long q = nbr3(g, v, p, 2 - t / 9, 2 - (t / 3) % 3, 2 - t % 3);
    if (q < 0) continue;
    const float2 d = dy[q];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = fmaf(ws[(0 * 16 + c) * T3 + t], d.x, fmaf(ws[(1 * 16 + c) * T3 + t], d.y, acc[c]));
  }
  float hv[16];
  unpack16(h2 + p * 16, hv);
#pragma unroll
  for (int c = 0; c < 16; ++c) dh2[p * 16 + c] = hv[c] > 0.f ? acc[c] : 0.f;
}

__global__ void k3_bwd2(Geom3 g, const float* __restrict__ dh2, const __nv_bfloat16* __restrict__ w2,
                        const __nv_bfloat16* __restrict__ h1, float* __restrict__ dh1) {
  __shared__ __align__(16) float ws[T3][16][16];      // [tap][out][in]
  for (int i = threadIdx.x; i < NP32; i += blockDim.x) {
    const int o = i / (16 * T3), c = (i / T3) % 16, t = i % T3;
    ws[t][o][c] = __bfloat162float(w2[i]);
  }
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= g.npix()) return;
  const Vox v = vox_of(g, p);
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.f;
  for (int t = 0; t < T3; ++t) {
    const long long q = nbr3(g, v, p, 2 - t / 9, 2 - (t / 3) % 3, 2 - t % 3);
    if (q < 0) continue;
    const float4* d4 = reinterpret_cast<const float4*>(dh2 + q * 16);
    float d[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 x = d4[i];
      d[4 * i] = x.x; d[4 * i + 1] = x.y; d[4 * i + 2] = x.z; d[4 * i + 3] = x.w;
    }
#pragma unroll
    for (int o = 0; o < 16; ++o) {
      const float4* wv = reinterpret_cast<const float4*>(&ws[t][o][0]);
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 w = wv[q4];
        acc[4 * q4 + 0] = fmaf(w.x, d[o], acc[4 * q4 + 0]);
        acc[4 * q4 + 1] = fmaf(w.y, d[o], acc[4 * q4 + 1]);
        acc[4 * q4 + 2] = fmaf(w.z, d[o], acc[4 * q4 + 2]);
        acc[4 * q4 + 3] = fmaf(w.w, d[o], acc[4 * q4 + 3]);
      }
    }
  }
  float hv[16];
  unpack16(h1 + p * 16, hv);
#pragma unroll
  for (int c = 0; c < 16; ++c) dh1[p * 16 + c] = hv[c] > 0.f ? acc[c] : 0.f;
}

// weight gradient: dw[o][c][t] += sum_p dout[p][o] in[c](p + (t - 1)).
// INKIND 0: input is bf16(scale r) (2 channels from float2); 1: bf16
// activations.  DKIND 0: dout is float2; 1: float[16].  A block takes 128
// voxels, their coordinates and dout staged in shared memory.
template <int CIN, int COUT, int INKIND, int DKIND>
__global__ void k3_wgrad(Geom3 g, const void* __restrict__ in, const void* __restrict__ dout, float* __restrict__ dw) {
  constexpr int NPAR = COUT * CIN * T3;
  constexpr int TP = 128;
  __shared__ float sd[TP * COUT];
  __shared__ Vox sv[TP];
  const long long p0 = (long long)blockIdx.x * TP;
  for (int i = threadIdx.x; i < TP * COUT; i += blockDim.x) {
    const long long p = p0 + i / COUT;
    const int o = i % COUT;
    float v = 0.f;
    if (p < g.npix()) {
      if (DKIND == 0) {
        const float2 d = reinterpret_cast<const float2*>(dout)[p];
        v = (o == 0) ? d.x : d.y;
      } else {
        v = reinterpret_cast<const float*>(dout)[p * COUT + o];
      }
    }
    sd[i] = v;
  }
  for (int i = threadIdx.x; i < TP; i += blockDim.x)
    if (p0 + i < g.npix()) sv[i] = vox_of(g, p0 + i);
  __syncthreads();
  const int np = (int)min((long long)TP, g.npix() - p0);
  for (int par = threadIdx.x; par < NPAR; par += blockDim.x) {
    const int o = par / (CIN * T3), rem = par % (CIN * T3), c = rem / T3, t = rem % T3;
    const int a = t / 9, b = (t / 3) % 3, e = t % 3;
    float acc = 0.f;
    for (int k = 0; k < np; ++k) {
      const long long q = nbr3(g, sv[k], p0 + k, a, b, e);
      if (q < 0) continue;
      float x;
      if (INKIND == 0) {
        const float2 v = reinterpret_cast<const float2*>(in)[q];
        x = bf(c == 0 ? v.x : v.y);
      } else {
        x = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(in)[q * CIN + c]);
      }
      acc = fmaf(sd[k * COUT + o], x, acc);
    }
    atomicAdd(&dw[par], acc);
  }
}

// the same over the warp-level MMA tile (the variant the batched kernel runs)
__global__ void __launch_bounds__(nettile::NT, NET_CTAS_PER_SM)
    k_net_fused_mma(Geom g, const float2* __restrict__ x, float scale, const __nv_bfloat16* __restrict__ wb,
                    float2* __restrict__ y, int accumulate) {
  using namespace nettile;
  extern __shared__ __align__(128) unsigned char fsm_raw[];
  unsigned char* base = fsm_raw + ((128 - (saddr(fsm_raw) & 127)) & 127);
  mmat::Ctx c;
  mmat::setup(c, base, base + PLANES_BYTES, wb);
  for (int i = threadIdx.x; i < PLANES_BYTES / 16; i += blockDim.x) reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  const int tiles_x = (g.W + TW - 1) / TW, tiles_y = (g.H + TH - 1) / TH;
  const long long ntiles = (long long)g.B * tiles_x * tiles_y;
  float2 xr[SPT];
  Tile cur = net_tile_of(g, x, y, tiles_x, tiles_y, blockIdx.x);
  if (blockIdx.x < ntiles) load_x(cur, xr);
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long nt = t + gridDim.x;
    const Tile next = net_tile_of(g, x, y, tiles_x, tiles_y, nt < ntiles ? nt : t);
    mmat::run_tile(c, cur, xr, scale, accumulate, nt < ntiles ? &next : nullptr);
    cur = next;
  }
}

__global__ void k_to_bf16(const float* w, __nv_bfloat16* wb, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16(w[i]);
}

inline int nblk(long long n) { return (int)((n + NTH - 1) / NTH); }

}  // namespace
}  // namespace csff

struct csff_net {
  int dim = 2;                   // 2: 3x3 network, 3: 3x3x3 network
  int nparam = csff::NPARAM;
  float* w = nullptr;            // FP32 master [nparam]
  float* m = nullptr;            // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* wb = nullptr;   // BF16 copy used by the kernels
  int step = 0;
  // scratch, grown on demand (pixels)
  long long cap = 0;
  __nv_bfloat16 *h1 = nullptr, *h2 = nullptr;
  float *dh1 = nullptr, *dh2 = nullptr;
  float2 *y = nullptr, *E = nullptr, *G = nullptr, *dy = nullptr;
  double* sums = nullptr;
  int cap_b = 0;
  float2* cpatch = nullptr;
  int* tcerr = nullptr;          // set when a tensor-core layer's wait ran out
};

namespace {

#define NK(call, what)                                                   \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return csff::cuda_fail(e_, what);             \
  } while (0)

csff_status ninvalid(const char* s) {
  csff::set_error(s);
  return CSFF_ERR_INVALID_ARG;
}

csff_status ensure_scratch(csff_net* N, long long npix, int B, bool train) {
  if (npix >= (1ll << 31)) return ninvalid("more than 2^31 pixels");
  if (npix > N->cap || (train && !N->dh1)) {
    for (void* p : {(void*)N->h1, (void*)N->h2, (void*)N->dh1, (void*)N->dh2, (void*)N->y, (void*)N->E,
                    (void*)N->G, (void*)N->dy})
      if (p) cudaFree(p);
    N->h1 = N->h2 = nullptr;
    N->dh1 = N->dh2 = nullptr;
    N->y = N->E = N->G = N->dy = nullptr;
    long long cap = std::max(npix, N->cap);
    NK(cudaMalloc((void**)&N->h1, sizeof(__nv_bfloat16) * 16 * cap), "net scratch");
    NK(cudaMalloc((void**)&N->h2, sizeof(__nv_bfloat16) * 16 * cap), "net scratch");
    NK(cudaMalloc((void**)&N->y, sizeof(float2) * cap), "net scratch");
    if (train) {
      NK(cudaMalloc((void**)&N->dh1, sizeof(float) * 16 * cap), "net scratch");
      NK(cudaMalloc((void**)&N->dh2, sizeof(float) * 16 * cap), "net scratch");
      NK(cudaMalloc((void**)&N->E, sizeof(float2) * cap), "net scratch");
      NK(cudaMalloc((void**)&N->G, sizeof(float2) * cap), "net scratch");
      NK(cudaMalloc((void**)&N->dy, sizeof(float2) * cap), "net scratch");
    }
    N->cap = cap;
  }
  if (B > N->cap_b) {
    if (N->sums) cudaFree(N->sums);
    if (N->cpatch) cudaFree(N->cpatch);
    NK(cudaMalloc((void**)&N->sums, sizeof(double) * 2 * B), "net sums");
    NK(cudaMalloc((void**)&N->cpatch, sizeof(float2) * B), "net patch constants");
    N->cap_b = B;
  }
  return CSFF_OK;
}

// layer by layer, keeping h1 and h2 for the backward pass (training)
csff_status forward_stored(csff_net* N, csff::Geom g, const float2* r, float2* y, int accumulate, cudaStream_t s) {
  using namespace csff;
  const long long np = g.npix();
  const __nv_bfloat16* w1 = N->wb;
  const __nv_bfloat16* w2 = N->wb + NP1;
  const __nv_bfloat16* w3 = N->wb + NP1 + NP2;
  {
    ProfScope ps(PF_MG32, s, 8.0 * np + 2.0 * 32 * np + 8.0 * np, 2.0 * 9 * (2 * 16 + 16 * 16 + 16 * 2) * np);
    k_conv1<<<nblk(np), NTH, 0, s>>>(g, r, w1, N->h1);
    NK(cudaFuncSetAttribute(k_conv_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, ctc::SMEM), "conv attribute");
    NK(cudaFuncSetAttribute(k_conv_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, ctc::SMEM), "conv attribute");
    const long long tiles = (np + ctc::TM - 1) / ctc::TM;
    const unsigned grid = (unsigned)std::min<long long>(tiles, 152 * ctc::CTAS_PER_SM);
    k_conv_tc<2><<<grid, 128, ctc::SMEM, s>>>(g, N->h1, w2, N->h2, nullptr, 0, N->tcerr);
    k_conv_tc<3><<<grid, 128, ctc::SMEM, s>>>(g, N->h2, w3, nullptr, y, accumulate, N->tcerr);
  }
  count_launch(3);
  NK(cudaGetLastError(), "net forward");
  return CSFF_OK;
}

// y = N(scale r) (accumulate: y += N(scale r)), the three layers fused
csff_status forward(csff_net* N, csff::Geom g, const float2* r, float scale, float2* y, int accumulate,
                    cudaStream_t s) {
  using namespace csff;
  const long long np = g.npix();
  const long long ntiles =
      (long long)g.B * ((g.W + nettile::TW - 1) / nettile::TW) * ((g.H + nettile::TH - 1) / nettile::TH);
  NK(cudaFuncSetAttribute(k_net_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, NET_SMEM), "net attribute");
  const unsigned grid = (unsigned)std::min<long long>(ntiles, 152 * NET_CTAS_PER_SM);
  {
    ProfScope ps(PF_MG32, s, (accumulate ? 24.0 : 16.0) * np, 2.0 * 9 * (2 * 16 + 16 * 16 + 16 * 2) * np);
    k_net_fused<<<grid, nettile::NT, NET_SMEM, s>>>(g, r, scale, N->wb, y, accumulate, N->tcerr);
  }
  count_launch();
  NK(cudaGetLastError(), "net forward");
  return CSFF_OK;
}

// the 3D network layer by layer, the activations kept in the scratch:
// y = N(scale r) (accumulate: y += N(scale r))
csff_status forward3(csff_net* N, csff::Geom3 g, const float2* r, float scale, float2* y, int accumulate,
                     cudaStream_t s) {
  using namespace csff;
  const long long np = g.npix();
  csff_status st = ensure_scratch(N, np, g.B, false);
  if (st != CSFF_OK) return st;
  {
    ProfScope ps(PF_MG32, s, 8.0 * np + 64.0 * np + (accumulate ? 16.0 : 8.0) * np,
                 2.0 * T3 * (2 * 16 + 16 * 16 + 16 * 2) * np);
    k3_conv1<<<nblk(np), NTH, 0, s>>>(g, r, scale, N->wb, N->h1);
    k3_conv2<<<nblk(np), NTH, 0, s>>>(g, N->h1, N->wb + NP31, N->h2);
    k3_conv3<<<nblk(np), NTH, 0, s>>>(g, N->h2, N->wb + NP31 + NP32, y, accumulate);
  }
  count_launch(3);
  NK(cudaGetLastError(), "3D net forward");
  return CSFF_OK;
}

csff_status loss_grad3(csff_net* N, csff::Geom3 g, const float2* r, const float2* q, const double* c_host, int margin,
                       float* loss_host, cudaStream_t s) {
  using namespace csff;
  const long long np = g.npix();
  csff_status st = ensure_scratch(N, np, g.B, true);
  if (st != CSFF_OK) return st;
  std::vector<float2> cp(g.B);
  for (int b = 0; b < g.B; ++b) cp[b] = make_float2((float)c_host[2 * b], (float)c_host[2 * b + 1]);
  NK(cudaMemcpyAsync(N->cpatch, cp.data(), sizeof(float2) * g.B, cudaMemcpyHostToDevice, s), "patch constants");
  NK(cudaMemsetAsync(N->sums, 0, sizeof(double) * 2 * g.B, s), "sums");
  NK(cudaMemsetAsync(N->grad, 0, sizeof(float) * NPARAM3, s), "grad");
  st = forward3(N, g, r, 1.f, N->y, 0, s);
  if (st != CSFF_OK) return st;
  const __nv_bfloat16* w2 = N->wb + NP31;
  const __nv_bfloat16* w3 = N->wb + NP31 + NP32;
  k3_loss1<<<nblk(np), NTH, 0, s>>>(g, N->y, r, q, N->cpatch, margin, N->E, N->sums);
  k3_loss2<<<nblk(np), NTH, 0, s>>>(g, N->E, N->sums, q, N->cpatch, N->G, N->dy, 0);
  k3_loss2<<<nblk(np), NTH, 0, s>>>(g, N->E, N->sums, q, N->cpatch, N->G, N->dy, 1);
  k3_bwd3<<<nblk(np), NTH, 0, s>>>(g, N->dy, w3, N->h2, N->dh2);
  k3_bwd2<<<nblk(np), NTH, 0, s>>>(g, N->dh2, w2, N->h1, N->dh1);
  const int wb_blocks = (int)((np + 127) / 128);
  k3_wgrad<16, 2, 1, 0><<<wb_blocks, NTH, 0, s>>>(g, N->h2, N->dy, N->grad + NP31 + NP32);
  k3_wgrad<16, 16, 1, 1><<<wb_blocks, NTH, 0, s>>>(g, N->h1, N->dh2, N->grad + NP31);
  k3_wgrad<2, 16, 0, 1><<<wb_blocks, NTH, 0, s>>>(g, r, N->dh1, N->grad);
  count_launch(8);
  NK(cudaGetLastError(), "3D net backward");
  if (loss_host) {
    std::vector<double> sums(2 * g.B);
    NK(cudaMemcpyAsync(sums.data(), N->sums, sizeof(double) * 2 * g.B, cudaMemcpyDeviceToHost, s), "loss");
    NK(cudaStreamSynchronize(s), "sync");
    double L = 0;
    for (int b = 0; b < g.B; ++b) L += sums[2 * b + 1] > 0 ? sums[2 * b] / sums[2 * b + 1] : 0.0;
    *loss_host = (float)(L / g.B);
  }
  return CSFF_OK;
}

// one Adam step on N->grad
csff_status adam_step(csff_net* N, float lr, cudaStream_t s) {
  N->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)N->step), c2 = 1.f - std::pow(b2, (float)N->step);
  csff::k_adam<<<(N->nparam + 255) / 256, 256, 0, s>>>(N->w, N->m, N->v, N->grad, N->wb, N->nparam, lr, b1, b2,
                                                       1e-8f, c1, c2);
  csff::count_launch();
  NK(cudaGetLastError(), "adam");
  return CSFF_OK;
}

// the same with the warp-level MMA tile
csff_status forward_mma(csff_net* N, csff::Geom g, const float2* r, float2* y, cudaStream_t s) {
  using namespace csff;
  const long long np = g.npix();
  const long long ntiles =
      (long long)g.B * ((g.W + nettile::TW - 1) / nettile::TW) * ((g.H + nettile::TH - 1) / nettile::TH);
  NK(cudaFuncSetAttribute(k_net_fused_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, NET_SMEM), "net attribute");
  const unsigned grid = (unsigned)std::min<long long>(ntiles, 152 * NET_CTAS_PER_SM);
  {
    ProfScope ps(PF_MG32, s, 16.0 * np, 2.0 * 9 * (2 * 16 + 16 * 16 + 16 * 2) * np);
    k_net_fused_mma<<<grid, nettile::NT, NET_SMEM, s>>>(g, r, 1.f, N->wb, y, 0);
  }
  count_launch();
  NK(cudaGetLastError(), "net forward");
  return CSFF_OK;
}

// loss and weight gradient (into N->grad) for a batch of patches
csff_status loss_grad(csff_net* N, csff::Geom g, const float2* r, const float2* q, const double* c_host, int margin,
                      float* loss_host, cudaStream_t s) {
  using namespace csff;
  const long long np = g.npix();
  csff_status st = ensure_scratch(N, np, g.B, true);
  if (st != CSFF_OK) return st;
  std::vector<float2> cp(g.B);
  for (int b = 0; b < g.B; ++b) cp[b] = make_float2((float)c_host[2 * b], (float)c_host[2 * b + 1]);
  NK(cudaMemcpyAsync(N->cpatch, cp.data(), sizeof(float2) * g.B, cudaMemcpyHostToDevice, s), "patch constants");
  NK(cudaMemsetAsync(N->sums, 0, sizeof(double) * 2 * g.B, s), "sums");
  NK(cudaMemsetAsync(N->grad, 0, sizeof(float) * NPARAM, s), "grad");
  st = forward_stored(N, g, r, N->y, 0, s);
  if (st != CSFF_OK) return st;
  const __nv_bfloat16* w2 = N->wb + NP1;
  const __nv_bfloat16* w3 = N->wb + NP1 + NP2;
  k_loss1<<<nblk(np), NTH, 0, s>>>(g, N->y, r, q, N->cpatch, margin, N->E, N->sums);
  k_loss2<<<nblk(np), NTH, 0, s>>>(g, N->E, N->sums, q, N->cpatch, N->G, N->dy, 0);
  k_loss2<<<nblk(np), NTH, 0, s>>>(g, N->E, N->sums, q, N->cpatch, N->G, N->dy, 1);
  k_bwd3<<<nblk(np), NTH, 0, s>>>(g, N->dy, w3, N->h2, N->dh2);
  k_bwd2<<<nblk(np), NTH, 0, s>>>(g, N->dh2, w2, N->h1, N->dh1);
  const int wb_blocks = (int)((np + 127) / 128);
  k_wgrad<16, 2, 1, 0><<<wb_blocks, NTH, 0, s>>>(g, N->h2, N->dy, N->grad + NP1 + NP2);
  k_wgrad<16, 16, 1, 1><<<wb_blocks, NTH, 0, s>>>(g, N->h1, N->dh2, N->grad + NP1);
  k_wgrad<2, 16, 0, 1><<<wb_blocks, NTH, 0, s>>>(g, r, N->dh1, N->grad);
  count_launch(8);
  NK(cudaGetLastError(), "net backward");
  if (loss_host) {
    std::vector<double> sums(2 * g.B);
    NK(cudaMemcpyAsync(sums.data(), N->sums, sizeof(double) * 2 * g.B, cudaMemcpyDeviceToHost, s), "loss");
    NK(cudaStreamSynchronize(s), "sync");
    double L = 0;
    for (int b = 0; b < g.B; ++b) L += sums[2 * b + 1] > 0 ? sums[2 * b] / sums[2 * b + 1] : 0.0;
    *loss_host = (float)(L / g.B);
  }
  return CSFF_OK;
}

}  // namespace

extern "C" {

static csff_status net_create(int dim, const float* w_host, csff_net** out) {
  if (!out) return ninvalid("out is NULL");
  *out = nullptr;
  csff_net* N = new csff_net();
  N->dim = dim;
  N->nparam = dim == 3 ? csff::NPARAM3 : csff::NPARAM;
  auto fail = [&](csff_status s) {
    csff_net_destroy(N);
    return s;
  };
  cudaError_t e;
  const size_t np = (size_t)N->nparam;
  if ((e = cudaMalloc((void**)&N->w, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMalloc((void**)&N->m, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMalloc((void**)&N->v, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMalloc((void**)&N->grad, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMalloc((void**)&N->wb, sizeof(__nv_bfloat16) * np)) != cudaSuccess ||
      (e = cudaMalloc((void**)&N->tcerr, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(N->tcerr, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(N->m, 0, sizeof(float) * np)) != cudaSuccess ||
      (e = cudaMemset(N->v, 0, sizeof(float) * np)) != cudaSuccess)
    return fail(csff::cuda_fail(e, "net allocation"));
  csff_status s = csff_net_set_weights(N, w_host);
  if (s != CSFF_OK) return fail(s);
  *out = N;
  return CSFF_OK;
}

void csff_net_destroy(csff_net* N) {
  if (!N) return;
  for (void* p : {(void*)N->w, (void*)N->m, (void*)N->v, (void*)N->grad, (void*)N->wb, (void*)N->h1, (void*)N->h2,
                  (void*)N->dh1, (void*)N->dh2, (void*)N->y, (void*)N->E, (void*)N->G, (void*)N->dy,
                  (void*)N->sums, (void*)N->cpatch, (void*)N->tcerr})
    if (p) cudaFree(p);
  delete N;
}

csff_status csff_net_create(const float* w_host, csff_net** out) { return net_create(2, w_host, out); }
csff_status csff_net_create3(const float* w_host, csff_net** out) { return net_create(3, w_host, out); }

int csff_net_num_params(void) { return csff::NPARAM; }
int csff_net_num_params3(void) { return csff::NPARAM3; }



csff_status csff_net_set_weights(csff_net* N, const float* w_host) {
  if (!N || !w_host) return ninvalid("NULL argument");
  const int np = N->nparam;
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(w_host[i])) return ninvalid("non-finite weight");
  NK(cudaMemcpy(N->w, w_host, sizeof(float) * np, cudaMemcpyHostToDevice), "set weights");
  csff::k_to_bf16<<<(np + 255) / 256, 256>>>(N->w, N->wb, np);
  csff::count_launch();
  NK(cudaMemset(N->m, 0, sizeof(float) * np), "reset moments");
  NK(cudaMemset(N->v, 0, sizeof(float) * np), "reset moments");
  N->step = 0;
  NK(cudaDeviceSynchronize(), "set weights");
  return CSFF_OK;
}

csff_status csff_net_get_weights(const csff_net* N, float* w_host) {
  if (!N || !w_host) return ninvalid("NULL argument");
  NK(cudaMemcpy(w_host, N->w, sizeof(float) * N->nparam, cudaMemcpyDeviceToHost), "get weights");
  return CSFF_OK;
}

csff_status csff_net_forward(csff_net* N, int B, int H, int W, const void* r_dev, void* y_dev, void* stream) {
  if (!N || !r_dev || !y_dev || B < 1 || H < 1 || W < 1) return ninvalid("bad forward arguments");
  if (N->dim != 2) return ninvalid("a 3D network: csff_net_forward3");
  csff::Geom g{B, H, W};
  if (g.npix() >= (1ll << 31)) return ninvalid("more than 2^31 pixels");
  csff_status s = forward(N, g, (const float2*)r_dev, 1.f, (float2*)y_dev, 0, (cudaStream_t)stream);
  if (s != CSFF_OK) return s;
  NK(cudaStreamSynchronize((cudaStream_t)stream), "sync");
  return csff::net_check(N);
}

csff_status csff_net_forward_mma(csff_net* N, int B, int H, int W, const void* r_dev, void* y_dev, void* stream) {
  if (!N || !r_dev || !y_dev || B < 1 || H < 1 || W < 1) return ninvalid("bad forward arguments");
  if (N->dim != 2) return ninvalid("a 3D network has no warp-level MMA variant");
  csff::Geom g{B, H, W};
  if (g.npix() >= (1ll << 31)) return ninvalid("more than 2^31 pixels");
  csff_status s = forward_mma(N, g, (const float2*)r_dev, (float2*)y_dev, (cudaStream_t)stream);
  if (s != CSFF_OK) return s;
  NK(cudaStreamSynchronize((cudaStream_t)stream), "sync");
  return CSFF_OK;
}

csff_status csff_net_loss_grad(csff_net* N, int B, int H, int W, const void* r_dev, const void* q_dev,
                               const double* c_host, int margin, float* loss_host, float* grad_host, void* stream) {
  if (!N || !r_dev || !q_dev || !c_host || B < 1 || H < 2 * margin + 1 || W < 2 * margin + 1 || margin < 0)
    return ninvalid("bad loss arguments");
  if (N->dim != 2) return ninvalid("a 3D network: csff_net_loss_grad3");
  if ((long long)B * H * W >= (1ll << 31)) return ninvalid("more than 2^31 pixels");
  cudaStream_t s = (cudaStream_t)stream;
  csff_status st = loss_grad(N, csff::Geom{B, H, W}, (const float2*)r_dev, (const float2*)q_dev, c_host, margin,
                             loss_host, s);
  if (st != CSFF_OK) return st;
  if (grad_host) {
    NK(cudaMemcpyAsync(grad_host, N->grad, sizeof(float) * csff::NPARAM, cudaMemcpyDeviceToHost, s), "grad");
    NK(cudaStreamSynchronize(s), "sync");
  }
  return CSFF_OK;
}

csff_status csff_net_train_step(csff_net* N, int B, int H, int W, const void* r_dev, const void* q_dev,
                                const double* c_host, int margin, float lr, float* loss_host, void* stream) {
  if (!(lr > 0.f)) return ninvalid("learning rate must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  csff_status st = csff_net_loss_grad(N, B, H, W, r_dev, q_dev, c_host, margin, loss_host, nullptr, stream);
  if (st != CSFF_OK) return st;
  return adam_step(N, lr, s);
}

csff_status csff_net_forward3(csff_net* N, int B, int Z, int H, int W, const void* r_dev, void* y_dev, void* stream) {
  if (!N || !r_dev || !y_dev || B < 1 || Z < 1 || H < 1 || W < 1) return ninvalid("bad forward arguments");
  if (N->dim != 3) return ninvalid("a 2D network: csff_net_forward");
  const csff::Geom3 g{B, Z, H, W};
  if (g.npix() >= (1ll << 31)) return ninvalid("more than 2^31 voxels");
  csff_status s = forward3(N, g, (const float2*)r_dev, 1.f, (float2*)y_dev, 0, (cudaStream_t)stream);
  if (s != CSFF_OK) return s;
  NK(cudaStreamSynchronize((cudaStream_t)stream), "sync");
  return CSFF_OK;
}

csff_status csff_net_loss_grad3(csff_net* N, int B, int Z, int H, int W, const void* r_dev, const void* q_dev,
                                const double* c_host, int margin, float* loss_host, float* grad_host, void* stream) {
  if (!N || !r_dev || !q_dev || !c_host || B < 1 || margin < 0 || Z < 2 * margin + 1 || H < 2 * margin + 1 ||
      W < 2 * margin + 1)
    return ninvalid("bad loss arguments");
  if (N->dim != 3) return ninvalid("a 2D network: csff_net_loss_grad");
  const csff::Geom3 g{B, Z, H, W};
  if (g.npix() >= (1ll << 31)) return ninvalid("more than 2^31 voxels");
  cudaStream_t s = (cudaStream_t)stream;
  csff_status st = loss_grad3(N, g, (const float2*)r_dev, (const float2*)q_dev, c_host, margin, loss_host, s);
  if (st != CSFF_OK) return st;
  if (grad_host) {
    NK(cudaMemcpyAsync(grad_host, N->grad, sizeof(float) * csff::NPARAM3, cudaMemcpyDeviceToHost, s), "grad");
    NK(cudaStreamSynchronize(s), "sync");
  }
  return CSFF_OK;
}

csff_status csff_net_train_step3(csff_net* N, int B, int Z, int H, int W, const void* r_dev, const void* q_dev,
                                 const double* c_host, int margin, float lr, float* loss_host, void* stream) {
  if (!(lr > 0.f)) return ninvalid("learning rate must be positive");
  csff_status st = csff_net_loss_grad3(N, B, Z, H, W, r_dev, q_dev, c_host, margin, loss_host, nullptr, stream);
  if (st != CSFF_OK) return st;
  return adam_step(N, lr, (cudaStream_t)stream);
}

}  // extern "C"

namespace csff {

const void* net_weights_bf16(const csff_net* N) { return N->wb; }
int net_dim(const csff_net* N) { return N->dim; }

// Before graph capture: the 2D network's inference keeps its activations in
// shared memory (only the 32-bit indexing limit to check); the 3D network's
// layers need their scratch for npix voxels.
csff_status net_reserve(csff_net* N, long long npix) {
  if (npix >= (1ll << 31)) return ninvalid("more than 2^31 pixels");
  return N->dim == 3 ? ensure_scratch(N, npix, 1, false) : CSFF_OK;
}

// status of the tensor-core layers since the last check (synchronises)
csff_status net_check(csff_net* N) {
  int err = 0;
  cudaError_t e = cudaMemcpy(&err, N->tcerr, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "net status");
  if (err) {
    cudaMemset(N->tcerr, 0, sizeof(int));
    set_error("learned smoother: a tensor-core wait ran out");
    return CSFF_ERR_TIMEOUT;
  }
  return CSFF_OK;
}

csff_status learned_step(csff_plan* P, int level, int dim, const Level& L, float2* u, const float2* b, cudaStream_t s) {
  csff_net* N = (level >= 0 && level < 16 && P->level_net[level]) ? P->level_net[level] : P->net;
  cudaError_t e = launch_residual<float>(dim, L, u, b, L.r32, s);
  if (e != cudaSuccess) return cuda_fail(e, "learned step residual");
  if (dim == 3) return forward3(N, Geom3{1, L.m, L.m, L.m}, L.r32, (float)(L.h * L.h), u, 1, s);
  Geom g{1, L.m, L.m};
  // u += N(h^2 r) = h^2 N(r) (the scaling applied as the input is read): the
  // network is positively homogeneous, and in units of h^2 the level's
  // operator e^{-2i gamma}(4 - shift) - (kh)^2 (1 + chi) is O(1) on every
  // grid, so one net serves levels with the same k h
  return forward(N, g, L.r32, (float)(L.h * L.h), u, 1, s);
}

}  // namespace csff
