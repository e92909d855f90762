// Internal declarations shared by the CUDA translation units of libcsff.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/csff.h"

namespace csff {

// ---------------------------------------------------------------------------
// complex helpers (interleaved re/im in CUDA vector types)
// ---------------------------------------------------------------------------
template <typename T> struct CxT;
template <> struct CxT<double> { using type = double2; };
template <> struct CxT<float> { using type = float2; };
template <typename T> using cx = typename CxT<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C{}.x) a, decltype(C{}.x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C, typename S> __host__ __device__ __forceinline__ C cscale(C a, S s) {
  return mk<C>(a.x * s, a.y * s);
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with launch_pdl is set up
// while its predecessor in the stream runs, and starts once every CTA of the
// predecessor has triggered its dependents (pdl_trigger) or exited.  The
// fused tiles trigger as they enter their last phase, so the next kernel's
// CTAs take the slots of retiring tiles; an explicit trigger at kernel start
// measured slower on the 1025^2 solves (early CTAs hold slots the
// predecessor's later waves need).  Every such kernel calls pdl_prologue(),
// which waits until the predecessor has completed and its writes are
// visible, before it touches anything the predecessor writes (the up tile
// first copies its iterate, right-hand side and factor windows, written by
// kernels that completed before the predecessor passed its own wait);
// launched the ordinary way, both are no-ops.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_prologue() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// plan internals
// ---------------------------------------------------------------------------
struct Level {
  int n = 0, m = 0;
  long long N = 0;       // m^d
  double h = 0;
  double2 c{};           // e^{-2i gamma} / h^2
  // per-point coefficients
  double2* q64 = nullptr;     // k^2 (1 + chi)
  double2* dinv64 = nullptr;  // 1 / (2d c - q)
  float2* q32 = nullptr;
  float2* dinv32 = nullptr;
  // separable factors of q for the FP32 fused tiles: [n_gauss][2][m],
  // X_g = 2^-s_g k^2 A_g e^{-(z_x-c_gx)^2/w_g}, Y_g = 2^s_g e^{-(z_y-c_gy)^2/w_g}
  float2* fac32 = nullptr;
  int ng = 0;
  double k2 = 0;
  // work buffers
  double2 *u64 = nullptr, *t64 = nullptr, *b64 = nullptr, *r64 = nullptr;
  float2 *u32 = nullptr, *t32 = nullptr, *b32 = nullptr, *r32 = nullptr;
};

// Far-field scratch (grown on demand): g = chi (u_in + u); x/y/z phase
// tables; stage-1 sums T; angle data; per-row exponents; misc[0] = max
// exponent of |g|, misc[1] = "a scale was applied" flag.
struct FFBuffers {
  size_t g = 0, xt = 0, yt = 0, zt = 0, T = 0, al = 0, ux = 0, xr = 0, s1 = 0;
  double2 *dg = nullptr, *dxt = nullptr, *dyt = nullptr, *dzt = nullptr, *dT = nullptr;
  double *dal = nullptr, *dux = nullptr;
  int *dxr = nullptr, *ds1 = nullptr, *dmisc = nullptr;
  // double-float stage 1: split operands, block exponents, spread flags [2]
  size_t xdf = 0, gdf = 0, exs = 0, egs = 0, xsm = 0, gsm = 0;
  float4 *dxdf = nullptr, *dgdf = nullptr;
  float2 *dxsm = nullptr, *dgsm = nullptr;   // re + im of the split operands
  int *dex = nullptr, *deg = nullptr, *dspread = nullptr;
  // block bounds for skipping negligible blocks and the per-tile skip flags
  size_t xlo = 0, ghi = 0, skip = 0;
  int *dxlo = nullptr, *dghi = nullptr;
  unsigned char* dskip = nullptr;
  size_t skip_used = 0;       // flags written by the last 2D far field
  // tensor-core 3D stage A: pre-swizzled split phase operand, per-column and
  // per-row exponents, [spread_g, spread_P, error word]
  size_t tcb = 0, tce = 0;
  unsigned char* dtcb = nullptr;
  int *dtce = nullptr, *dtcflag = nullptr;
};

// Device state of one GMRES(m) smoothing step (gmres.cu): the (m+1) x m
// Hessenberg matrix, the norms beta = nrm[0] and h_{j+1,j} = nrm[j+1] with their
// inverses, the least-squares solution y and the number k of columns used.
constexpr int GM_MAX = 4;
struct GmState {
  double2 H[GM_MAX + 1][GM_MAX];
  double nrm[GM_MAX + 1];
  double inv[GM_MAX + 1];
  double2 y[GM_MAX];
  int k;
};

}  // namespace csff

struct csff_plan {
  csff_problem prob{};
  int ff_mode = 0;          // CSFF_FF_FP64 or CSFF_FF_TC_BF16X4
  std::vector<csff_gauss> gauss;
  csff_opts opts{};
  cudaStream_t stream = nullptr;
  int dim = 2;
  std::vector<csff::Level> lv;
  // separable tables of chi per level: [n_gauss][dim][m_l] (amplitude folded
  // into axis 0), FP64 on the device
  std::vector<double2*> chi_tab;
  double2* coarse_inv = nullptr;  // dense inverse of the coarsest operator (FP64 Gauss-Jordan)
  float2* coarse_inv32 = nullptr;  // the same inverse rounded to FP32, applied in FP32 cycles
  int coarse_N = 0;
  // per-solve data
  double2* uinc_tab = nullptr;    // [dim][m] for the current eta
  double* red = nullptr;          // reduction partials
  double* red_out = nullptr;      // device scalars (norms)
  double* red_host = nullptr;     // pinned host mirror
  int red_blocks = 0;
  csff::FFBuffers ff;
  size_t bytes = 0;
  double log_rhs_max = 0, log_ff_max = 0;
  // fused V(1,1) RB-GS path (2D): levels >= fused_lc run in one CTA; -1 = unfused
  int fused_lc = -1;
  // CUDA graphs of solver steps (FP64 cycle, or mixed refinement step of a
  // given cycle count), captured on an internal stream and kept by key; the
  // oldest is replaced when all slots are taken
  static constexpr int GRAPH_SLOTS = 8;
  struct StepGraph {
    long long key = 0;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;         // kernel nodes in the captured graph
  };
  StepGraph graphs[GRAPH_SLOTS];
  int graph_next = 0;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev = nullptr;
  bool use_graphs = true;
  // learned smoother (csff_plan_set_learned): RB-GS sweep followed by
  // u += N(r) on levels < learned_levels of the FP32 cycles
  csff_net* net = nullptr;
  csff_net* level_net[16] = {};   // per-level replacements of net (csff_plan_set_learned_level)
  int learned_levels = 0;
  double learned_guard = 0.5;
  bool learned_off = false;       // per-solve fallback to plain RB-GS
  // GMRES(m) smoother: m+1 basis vectors of the finest level (sized for FP64,
  // shared by every level and both precisions), reduction partials, state
  void* gm_v = nullptr;
  double2* gm_part = nullptr;
  csff::GmState* gm = nullptr;
  // coefficients from user samples (csff_plan_set_potential) and the scratch
  // of csff_separable_sum
  bool user_q = false;
  double2* sep_T = nullptr;
  size_t sep_cap = 0;
  // mixed refinement in double-float (refine_df.cu): iterate, right-hand side
  // and coefficients of the finest level as (re hi, re lo, im hi, im lo)
  float4 *dfu = nullptr, *dfb = nullptr, *dfq = nullptr;
  bool dfq_ready = false;
  double* dfpart = nullptr;     // per-block partial sums of |r'|^2
  int refine_eb = 0;            // FP64 refinement: the right-hand side's exponent of this solve

};

namespace csff {

// error reporting (thread-local last error)
void set_error(const std::string& s);
csff_status cuda_fail(cudaError_t e, const char* what);
extern std::atomic<uint64_t> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Event bracket around the launches of one kernel family (see csff_prof_begin).
enum ProfFamily { PF_FF_CONTRACT = 0, PF_MG32 = 1, PF_MG64 = 2, PF_FF_OTHER = 3, PF_TILES32 = 4, PF_TILES32_FINE = 5 };
// events around one launch, counted in family and (when >= 0) in family2 as well
// The adaptive refinement schedule (csff_refinement_cycles), shared by the
// host (single plans) and the batched kernel: after a step of cycles_run FP32
// V-cycles took the relative residual from rel_before to rel_after, the next
// step runs ceil(log(rel_tol / rel_after) / log rho) cycles, rho the step's
// per-cycle factor, clamped to [1, max_cycles]; max_cycles without a reduction.
__host__ __device__ inline int refinement_cycles(double rel_before, double rel_after, int cycles_run,
                                                 double rel_tol, int max_cycles) {
  const int cap = max_cycles > 1 ? max_cycles : 1;
  if (!(rel_after > 0.0) || !(rel_before > rel_after) || !isfinite(rel_before) || !(rel_tol > 0.0) ||
      cycles_run < 1)
    return cap;
  if (rel_after <= rel_tol) return 1;
  const double rho = pow(rel_after / rel_before, 1.0 / cycles_run);
  if (!(rho > 0.0) || !(rho < 1.0)) return cap;
  // 1e-9 of slack keeps a ratio that is an integer up to rounding from taking one
  // cycle more
  const double need = ceil(log(rel_tol / rel_after) / log(rho) - 1e-9);
  if (!(need < cap)) return cap;
  return need < 1.0 ? 1 : (int)need;
}

struct ProfScope {
  int slot = -1, slot2 = -1, slot3 = -1;
  cudaStream_t stream = nullptr;
  ProfScope(int family, cudaStream_t s, double bytes, double flops, int family2 = -1, int family3 = -1);
  ~ProfScope();
};
template <typename T> constexpr int mg_family() { return sizeof(T) == 8 ? PF_MG64 : PF_MG32; }

// ---- multigrid kernel launchers (mg_kernels.cu) ----------------------------
template <typename T>
cudaError_t launch_residual(int dim, const Level& L, const cx<T>* u, const cx<T>* b, cx<T>* r,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_jacobi(int dim, const Level& L, double omega, const cx<T>* u, const cx<T>* b,
                          cx<T>* u_out, cudaStream_t s);
template <typename T>
cudaError_t launch_rbgs(int dim, const Level& L, cx<T>* u, const cx<T>* b, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(int dim, const Level& F, const Level& C, const cx<T>* r, cx<T>* bc,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_prolong_add(int dim, const Level& F, const Level& C, const cx<T>* ec, cx<T>* u,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve(const cx<T>* inv, int N, const cx<T>* b, cx<T>* u, cudaStream_t s);
// FP32 vectors, FP64 inverse and product, one rounding of the result to FP32
cudaError_t launch_coarse_solve_f64(const double2* inv, int N, const float2* b, float2* u, cudaStream_t s);
// ||v||_2 * 2^{-e_scale}... computed as sqrt(sum |v 2^-e|^2) * 2^e; result to out (device)
template <typename T>
cudaError_t launch_norm2(const cx<T>* v, long long N, int exp_scale, double* partial, int nblk,
                         double* out, cudaStream_t s);
// max exponent (frexp) of |v| over N values -> *out (device int)
cudaError_t launch_max_exp(const double2* v, long long N, int* out, cudaStream_t s);
cudaError_t launch_coefs(int dim, const Level& L, const double2* const* chi_tab, int n_gauss,
                         double k2, cudaStream_t s);
cudaError_t launch_rhs(int dim, int m, const double2* const* chi_tab, int n_gauss,
                       const double2* uinc_tab, double k2, double2* b, cudaStream_t s);
template <typename T>
cudaError_t launch_zero(cx<T>* v, long long N, cudaStream_t s);

// q_c = q_f at the coarse nodes (injection), then 1/d, q and 1/d in FP32 from
// each level's q64 (csff_plan_set_potential)
cudaError_t launch_inject_q(int dim, const Level& F, const Level& C, cudaStream_t s);
cudaError_t launch_coefs_from_q(int dim, const Level& L, cudaStream_t s);
// out = a + s v (complex v, real a and s) over N values (partial_wave.cu: the
// Schroedinger coefficients q = 2E - 2V and right-hand side 2 phi)
cudaError_t launch_affine(const double2* v, long long N, double a, double s, double2* out, cudaStream_t st);

// ---- double-float refinement (refine_df.cu) -------------------------------------
// out = 2^exp_scale v split into float pairs; r = b - A u in double-float, rounded
// to FP32; u += e with TwoSum; out = 2^exp_scale (hi + lo)
// out = v 2^exp_scale as double-float pairs; r32 (optional): the same rounded to
// FP32; norm_out (optional): ||r32||, with part holding df_split_blocks doubles
cudaError_t launch_df_split(const double2* v, long long N, int exp_scale, float4* out, float2* r32, double* part,
                            double* norm_out, cudaStream_t s);
long long df_split_blocks(long long N);
long long df_residual_blocks(int dim, int m);
// r = b' - A u' rounded to FP32; with norm_out, also ||r|| (part: one double
// per block of the residual kernel, df_residual_blocks of them)
cudaError_t launch_df_residual(int dim, const Level& L, const float4* u, const float4* b, const float4* q,
                               float2* r, double* part, double* norm_out, cudaStream_t s);
cudaError_t launch_df_update(float4* u, const float2* e, long long N, cudaStream_t s);
cudaError_t launch_df_to64(const float4* u, long long N, int exp_scale, double2* out, cudaStream_t s);

// ---- FP64 refinement of the mixed solve (option refine_fp64; mg_kernels.cu) ------
// r32 = 2^-e r with e the exponent of *norm_dev (written to *exp_out); u += 2^e e32
cudaError_t launch_to32_scaled(const double2* r, long long N, const double* norm_dev, float2* r32,
                               int* exp_out, cudaStream_t s);
cudaError_t launch_update64(double2* u, const float2* e, long long N, const int* exp_in, cudaStream_t s);
// The FP64 refinement step with a fixed scale 2^s: r = b - A u in FP64, r32 =
// 2^-s r in FP32, ||r|| into *out (device; partial: nblk doubles of scratch);
// u += 2^s e; r32 = 2^-s v.  N < 2^31.
cudaError_t launch_refine_residual(int dim, const Level& L, const double2* u, const double2* b, int s_exp,
                                   float2* r32, double* partial, int nblk, double* out, cudaStream_t s);
cudaError_t launch_update64_fixed(double2* u, const float2* e, long long N, int s_exp, cudaStream_t s);
cudaError_t launch_scale_to32(const double2* v, long long N, int s_exp, float2* r32, cudaStream_t s);

// ---- GMRES(m) smoothing step (gmres.cu) ----------------------------------------
// u += V y for the GMRES(m) minimiser from u; V holds m+1 vectors of L.N
// values, part at least part_cap double2 partial sums, S the step's state.
template <typename T>
cudaError_t launch_gmres_step(int dim, const Level& L, int m, cx<T>* u, const cx<T>* b, cx<T>* V,
                              double2* part, int part_cap, GmState* S, cudaStream_t s);

// ---- fused 2D V(1,1) RB-GS kernels (mg_fused.cu) ----------------------------
size_t coarse_levels_smem(int dim, const std::vector<Level>& lv, int lc, int real_bytes);
// finest: the launch works on the plan's finest level (a profiling family of its own)
template <typename T>
cudaError_t launch_down2(const Level& F, const Level& Cl, const cx<T>* u_in, bool zero_init, const cx<T>* b,
                         cx<T>* u_out, cx<T>* bc, cudaStream_t s, bool finest = false);
template <typename T>
cudaError_t launch_up2(const Level& F, const Level& Cl, const cx<T>* u_in, const cx<T>* ec, const cx<T>* b,
                       cx<T>* u_out, cudaStream_t s, bool finest = false);
// inv64 (FP32 cycles only, may be null): the FP64 inverse, applied in FP64
// to the coarsest right-hand side in place of inv
template <typename T>
cudaError_t launch_coarse_levels(int dim, const std::vector<Level>& lv, int lc, const cx<T>* inv,
                                 const double2* inv64, const cx<T>* b, cx<T>* u, cudaStream_t s);
// dynamic shared-memory opt-in of the fused kernels on the current device
cudaError_t prepare_fused(int dim, const std::vector<Level>& lv, int lc);
// true while a graph is being captured (profiling brackets are suppressed)
extern thread_local bool g_capturing;
// kernel families currently timed (csff_prof_begin mask)
unsigned prof_mask();

// ---- learned smoother (learned.cu) ------------------------------------------
csff_status learned_step(csff_plan* P, int level, int dim, const Level& L, float2* u, const float2* b, cudaStream_t s);
csff_status net_reserve(csff_net* N, long long npix);
csff_status net_check(csff_net* N);
const void* net_weights_bf16(const csff_net* N);   // the network's BF16 weights on the device
int net_dim(const csff_net* N);                    // 2 or 3

// ---- far field (farfield.cu) -----------------------------------------------
void free_ff_buffers(csff_plan* P);
csff_status far_field_executed(csff_plan* P, double* executed);
csff_status far_field_one(csff_plan* P, const double* eta_host, const double2* u, int n_ang,
                          const double* alpha_host, double2* F, int32_t* F_exp, bool* scaled);

}  // namespace csff
