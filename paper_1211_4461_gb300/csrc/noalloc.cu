// Allocation-free variant of the Euclidean-norm reduction (csff_norm2_noalloc).
//
// Some callers cannot allocate device memory: code whose device memory is
// owned by another allocator (a framework's caching allocator, a
// pre-reserved arena) and loops that must not pay cudaMalloc's implicit
// device synchronisation.  This entry point needs no plan and allocates
// nothing: its per-block partial sums live in a file-scope device array of
// fixed size, which every GPU that loads the library holds until exit.
//
// The host cannot use the array's name as a device address, so the first call
// on each device looks the address up with cudaGetSymbolAddress (that device
// current) and caches it together with the id of the CUDA context it belongs
// to; later calls on that device reuse it while the context is the same.  A
// new context on the device (after cudaDeviceReset, for instance) holds a new
// copy of the array, so the address is looked up again.
#include <cuda.h>

#include <mutex>

#include "csff_internal.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 32;                   // elements per thread, no grid stride
constexpr int NA_MAX_PARTIALS = 4096;          // one partial per block
constexpr long long NA_MAX_N = (long long)NA_MAX_PARTIALS * NA_THREADS * NA_ITEMS;  // 2^25
constexpr int NA_MAX_DEVICES = 64;

// Shared by every call: the partials of the last call stay here until the next
// call overwrites them.  Each block writes its own partial before the finishing
// kernel reads it, so nothing needs clearing.
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_PARTIALS];

template <typename T>
__global__ void k_na_partial(const csff::cx<T>* __restrict__ v, long long n, double scale,
                             double* __restrict__ partial) {
  __shared__ double sh[NA_THREADS / 32];
  const long long base = (long long)blockIdx.x * NA_THREADS * NA_ITEMS + threadIdx.x;
  double acc = 0;
#pragma unroll 4
  for (int i = 0; i < NA_ITEMS; ++i) {
    long long j = base + (long long)i * NA_THREADS;
    if (j < n) {
      double a = (double)v[j].x * scale, b = (double)v[j].y * scale;
      acc = fma(a, a, fma(b, b, acc));
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < NA_THREADS / 32; ++w) s += sh[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_na_finish(const double* __restrict__ partial, int nblk, double inv_scale,
                            double* __restrict__ out) {
  __shared__ double sh[NA_THREADS / 32];
  double acc = 0;
  for (int i = threadIdx.x; i < nblk; i += NA_THREADS) acc += partial[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < NA_THREADS / 32; ++w) s += sh[w];
    *out = sqrt(s) * inv_scale;
  }
}

std::mutex g_na_mutex;
double* g_na_addr[NA_MAX_DEVICES] = {nullptr};
unsigned long long g_na_ctx[NA_MAX_DEVICES] = {0};

// Id of the calling thread's current CUDA context (0 if none is current or the
// driver cannot tell).  The two driver calls are fetched through the runtime,
// so the library does not link against the driver library.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, nullptr) == cudaSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, nullptr) == cudaSuccess)
      get_id = reinterpret_cast<GetId>(f);
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the partials array on the current device: looked up on
// the first call on the device and again whenever its context has changed.
cudaError_t partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  const unsigned long long ctx = current_context_id();
  if (!g_na_addr[dev] || ctx == 0 || ctx != g_na_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);   // makes the device's context current if needed
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = static_cast<double*>(p);
    g_na_ctx[dev] = current_context_id();
  }
  *out = g_na_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" csff_status csff_norm2_noalloc(int arith, const void* v_dev, long long n, int exp_scale,
                                          double* out_dev, void* stream) {
  if (arith != CSFF_ARITH_FP64 && arith != CSFF_ARITH_FP32) {
    csff::set_error("csff_norm2_noalloc: arith must be CSFF_ARITH_FP64 or CSFF_ARITH_FP32");
    return CSFF_ERR_INVALID_ARG;
  }
  if (!v_dev || !out_dev || n < 0) {
    csff::set_error("csff_norm2_noalloc: NULL pointer or negative length");
    return CSFF_ERR_INVALID_ARG;
  }
  if (n > NA_MAX_N) {
    csff::set_error("csff_norm2_noalloc: n exceeds the fixed scratch limit of 33554432 values");
    return CSFF_ERR_INVALID_ARG;
  }
  if (exp_scale < -1000 || exp_scale > 1000) {
    csff::set_error("csff_norm2_noalloc: exp_scale must lie in [-1000, 1000]");
    return CSFF_ERR_INVALID_ARG;
  }
  double* partials = nullptr;
  cudaError_t e = partials_address(&partials);
  if (e != cudaSuccess) return csff::cuda_fail(e, "csff_norm2_noalloc: scratch address");
  cudaStream_t s = (cudaStream_t)stream;
  const long long per_block = (long long)NA_THREADS * NA_ITEMS;
  int nblk = (int)((n + per_block - 1) / per_block);
  if (nblk < 1) nblk = 1;
  const double scale = ldexp(1.0, -exp_scale), inv = ldexp(1.0, exp_scale);
  if (arith == CSFF_ARITH_FP64)
    k_na_partial<double><<<nblk, NA_THREADS, 0, s>>>((const double2*)v_dev, n, scale, partials);
  else
    k_na_partial<float><<<nblk, NA_THREADS, 0, s>>>((const float2*)v_dev, n, scale, partials);
  k_na_finish<<<1, NA_THREADS, 0, s>>>(partials, nblk, inv, out_dev);
  csff::count_launch(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return csff::cuda_fail(e, "csff_norm2_noalloc: launch");
  return CSFF_OK;
}
