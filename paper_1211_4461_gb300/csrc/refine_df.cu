// The outer refinement of the mixed solve in double-float arithmetic.
//
// Mixed refinement: r = b - A u, an FP32 V-cycle solve of A e = r, u += e,
// repeated until ||r|| <= rel_tol ||b||.  The residual must be formed more
// accurately than the FP32 cycles work, but FP64 runs at 1/61 of the FP32 rate
// on this part, and the FP64 residual of a 1025^2 map costs about 46 us.  Here
// the iterate u, the right-hand side b and the coefficients q are held as
// pairs of floats hi + lo (48 significant bits), all scaled by 2^-e_b (e_b:
// the exponent of max |b|, so every value lies inside the FP32 range), and
// the residual r' = b' - A u' is formed with error-free transformations on the
// FP32 pipes: TwoSum for sums, an FMA-based TwoProd for products.  Its error,
// about 2^-46 (|c| |2d u - sum_nbr u| + |q u|) per point, stays six orders of
// magnitude under a 1e-8 residual.  The residual is written rounded to FP32 -
// the accuracy the FP32 cycles use - straight into their right-hand side: the
// V-cycle is linear and bias-free, so no further scaling is needed, and the
// correction it returns is added to u' with TwoSum.  The splits of b, q and the
// initial guess work on the IEEE fields (df_bits.cuh); FP64 arithmetic is left
// only in assembling u = 2^e_b (hi + lo) once per solve.  The classical form,
// with the residual and update in FP64, stays available as the option
// refine_fp64 (mg_kernels.cu).
#include <cmath>

#include "csff_internal.h"
#include "df_bits.cuh"

namespace csff {
namespace {

constexpr int BX = 32, BY = 8;

struct dff {
  float hi, lo;
};

// The transformations below rely on every sum and product being rounded on its
// own: the _rn intrinsics keep the compiler from contracting a product and the
// sum that follows it into one FMA, which would break TwoSum's identity.
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ dff two_sum(float a, float b) {
  const float s = add(a, b), bb = sub(s, a);
  return dff{s, add(sub(a, sub(s, bb)), sub(b, bb))};
}
__device__ __forceinline__ dff renorm(float s, float e) {
  const float h = add(s, e);
  return dff{h, sub(e, sub(h, s))};
}
__device__ __forceinline__ dff dadd(dff x, dff y) {
  const dff s = two_sum(x.hi, y.hi);
  return renorm(s.hi, add(s.lo, add(x.lo, y.lo)));
}
__device__ __forceinline__ dff dneg(dff x) { return dff{-x.hi, -x.lo}; }
__device__ __forceinline__ dff dmul(dff x, dff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);          // exact error of the leading product
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return renorm(p, e);
}
// s a power of two: exact
__device__ __forceinline__ dff dscale(dff x, float s) { return dff{__fmul_rn(x.hi, s), __fmul_rn(x.lo, s)}; }

struct cdf {
  dff re, im;
};
__device__ __forceinline__ cdf load(const float4* p, long long i) {
  const float4 v = p[i];
  return cdf{dff{v.x, v.y}, dff{v.z, v.w}};
}
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cdf{dadd(a.re, b.re), dadd(a.im, b.im)}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cdf{dadd(a.re, dneg(b.re)), dadd(a.im, dneg(b.im))}; }
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  return cdf{dadd(dmul(a.re, b.re), dneg(dmul(a.im, b.im))), dadd(dmul(a.re, b.im), dmul(a.im, b.re))};
}

// out = (re hi, re lo, im hi, im lo) of v 2^-e; r32 (optional) = v 2^-e rounded
// to FP32, i.e. the residual b' - A 0 when v is the right-hand side; part
// (optional): per block, the sum of |r32|^2 (FP32 squares summed in FP64)
__global__ void k_df_split(const double2* __restrict__ v, long long N, int e, float4* __restrict__ out,
                           float2* __restrict__ r32, double* __restrict__ part) {
  pdl_prologue();
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 x = v[i];
    const float2 re = bits::split_scaled(x.x, e), im = bits::split_scaled(x.y, e);
    out[i] = make_float4(re.x, re.y, im.x, im.y);
    if (r32) r32[i] = make_float2(re.x, im.x);
    if (part) acc += (double)fmaf(re.x, re.x, im.x * im.x);
  }
  if (!part) return;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

// r' = b' - (c (2d u' - sum_nbr u') - q u'), rounded to FP32.  part (optional):
// per block, the sum of |r'|^2 over its points (FP32 squares and warp sums,
// FP64 across warps): the squares of FP32 residual entries stay normal down to
// entries of 1e-19, far below any tolerance relative to max |b'| in [1/2, 1).
template <int D>
__device__ __forceinline__ float2 df_residual_point(const float4* __restrict__ u, const float4* __restrict__ b,
                                                   const float4* __restrict__ q, float4 c4, int m, int ix, int iy,
                                                   int iz, long long idx) {
  const cdf zero{dff{0.f, 0.f}, dff{0.f, 0.f}};
  cdf s = zero;
  if (ix > 0) s = cadd(s, load(u, idx - 1));
  if (ix < m - 1) s = cadd(s, load(u, idx + 1));
  if (iy > 0) s = cadd(s, load(u, idx - m));
  if (iy < m - 1) s = cadd(s, load(u, idx + m));
  if (D == 3) {
    const long long p = (long long)m * m;
    if (iz > 0) s = cadd(s, load(u, idx - p));
    if (iz < m - 1) s = cadd(s, load(u, idx + p));
  }
  const cdf uj = load(u, idx);
  // 2d u: a power-of-two scale in 2D, an exact product (TwoProd) for 6 in 3D
  const cdf ud = (D == 2) ? cdf{dscale(uj.re, 4.f), dscale(uj.im, 4.f)}
                          : cdf{dmul(uj.re, dff{6.f, 0.f}), dmul(uj.im, dff{6.f, 0.f})};
  const cdf t = csub(ud, s);
  const cdf c{dff{c4.x, c4.y}, dff{c4.z, c4.w}};
  const cdf au = csub(cmul(c, t), cmul(load(q, idx), uj));
  const cdf rr = csub(load(b, idx), au);
  return make_float2(add(rr.re.hi, rr.re.lo), add(rr.im.hi, rr.im.lo));
}

template <int D>
__global__ void k_df_residual(const float4* __restrict__ u, const float4* __restrict__ b,
                              const float4* __restrict__ q, float4 c4, int m, float2* __restrict__ r,
                              double* __restrict__ part) {
  pdl_prologue();
  const int ix = blockIdx.x * BX + threadIdx.x, iy = blockIdx.y * BY + threadIdx.y;
  const int iz = (D == 3) ? (int)blockIdx.z : 0;
  float sq = 0.f;
  if (ix < m && iy < m) {
    const long long idx = ((long long)iz * m + iy) * m + ix;
    const float2 v = df_residual_point<D>(u, b, q, c4, m, ix, iy, iz, idx);
    r[idx] = v;
    sq = fmaf(v.x, v.x, v.y * v.y);
  }
  if (!part) return;
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  __shared__ float ws[BX * BY / 32];
  const int t = threadIdx.y * BX + threadIdx.x;
  if ((t & 31) == 0) ws[t >> 5] = sq;
  __syncthreads();
  if (t == 0) {
    double acc = 0.0;
    for (int w = 0; w < BX * BY / 32; ++w) acc += (double)ws[w];
    part[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
  }
}

// out = sqrt(sum of the n partial sums)
__global__ void k_df_norm_finish(const double* __restrict__ part, long long n, double* __restrict__ out) {
  pdl_prologue();
  __shared__ double ws[32];
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    *out = sqrt(t);
  }
}

// u' += e (TwoSum per component)
__global__ void k_df_update(float4* __restrict__ u, const float2* __restrict__ e, long long N) {
  pdl_prologue();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const float4 v = u[i];
    const float2 d = e[i];
    const dff a = two_sum(v.x, d.x), bq = two_sum(v.z, d.y);
    const dff x = renorm(a.hi, add(a.lo, v.y)), y = renorm(bq.hi, add(bq.lo, v.w));
    u[i] = make_float4(x.hi, x.lo, y.hi, y.lo);
  }
}

// out = 2^e (hi + lo): the scale goes into the exponents of the widened words
__global__ void k_df_to64(const float4* __restrict__ u, long long N, int e, double2* __restrict__ out) {
  pdl_prologue();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const float4 v = u[i];
    out[i] = make_double2(bits::widen(v.x, e) + bits::widen(v.y, e), bits::widen(v.z, e) + bits::widen(v.w, e));
  }
}

int flat(long long N) {
  const long long b = (N + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

cudaError_t launch_df_split(const double2* v, long long N, int exp_scale, float4* out, float2* r32, double* part,
                            double* norm_out, cudaStream_t s) {
  if (norm_out && !part) return cudaErrorInvalidValue;
  cudaError_t e = launch_pdl(k_df_split, dim3(flat(N)), dim3(256), 0, s, v, N, -exp_scale, out, r32,
                             norm_out ? part : nullptr);
  count_launch();
  if (e == cudaSuccess && norm_out) {
    e = launch_pdl(k_df_norm_finish, dim3(1), dim3(512), 0, s, (const double*)part, (long long)flat(N), norm_out);
    count_launch();
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

long long df_split_blocks(long long N) { return flat(N); }

long long df_residual_blocks(int dim, int m) {
  return (long long)((m + BX - 1) / BX) * ((m + BY - 1) / BY) * (dim == 3 ? m : 1);
}

cudaError_t launch_df_residual(int dim, const Level& L, const float4* u, const float4* b, const float4* q,
                               float2* r, double* part, double* norm_out, cudaStream_t s) {
  // c = e^{-2 i gamma} / h^2 as two double-float parts
  const float cxh = (float)L.c.x, cyh = (float)L.c.y;
  const float4 c4 = make_float4(cxh, (float)(L.c.x - (double)cxh), cyh, (float)(L.c.y - (double)cyh));
  const dim3 g((L.m + BX - 1) / BX, (L.m + BY - 1) / BY, dim == 3 ? L.m : 1), blk(BX, BY);
  if (norm_out && !part) return cudaErrorInvalidValue;
  ProfScope ps(PF_MG64, s, 56.0 * L.N, 0);
  cudaError_t e = (dim == 2) ? launch_pdl(k_df_residual<2>, g, blk, 0, s, u, b, q, c4, L.m, r, part)
                             : launch_pdl(k_df_residual<3>, g, blk, 0, s, u, b, q, c4, L.m, r, part);
  count_launch();
  if (e == cudaSuccess && norm_out) {
    e = launch_pdl(k_df_norm_finish, dim3(1), dim3(512), 0, s, (const double*)part,
                   df_residual_blocks(dim, L.m), norm_out);
    count_launch();
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_df_update(float4* u, const float2* e, long long N, cudaStream_t s) {
  ProfScope ps(PF_MG64, s, 40.0 * N, 0);
  const cudaError_t r = launch_pdl(k_df_update, dim3(flat(N)), dim3(256), 0, s, u, e, N);
  count_launch();
  return r != cudaSuccess ? r : cudaGetLastError();
}

cudaError_t launch_df_to64(const float4* u, long long N, int exp_scale, double2* out, cudaStream_t s) {
  const cudaError_t e = launch_pdl(k_df_to64, dim3(flat(N)), dim3(256), 0, s, u, N, exp_scale, out);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace csff
