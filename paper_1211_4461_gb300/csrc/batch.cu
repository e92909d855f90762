// Batched solve of many uneven 2D problems in one persistent launch.
//
// Every instance runs the FP32-inner / FP64-refinement iteration of the
// single-problem path (FP64 residual, power-of-two scaled FP32 V(1,1) RB-GS
// cycles on the correction equation with the coarsest solve in FP64, FP64
// update), but all instances advance
// together inside ONE cooperative kernel: the iteration is a fixed sequence of
// phases (rhs, norms, scale to FP32, per-level down tiles, coarse block,
// per-level up tiles, update + residual, convergence), separated by grid
// barriers.  In each phase the CTAs share out the tiles of every active
// instance through prefix tables, so large and small grids run side by side.
// Convergence, divergence and non-finite checks are taken per instance on the
// device; converged instances drop out of the following phases.
//
// With a learned smoother (csff_batch_set_learned) every FP32 cycle of an
// instance ends with the learned step on its finest level, u <- u + N(h^2 r)
// with r = b - A u: a residual phase, then the network phase, whose work items
// are the 32 x 16 output tiles of the fused three-layer network (net_tile.cuh)
// of every instance that takes the step.  As in the single-problem solve the
// first two refinement steps of an instance run without it, the second sets
// the reference reduction factor (at most the guard), and an instance whose
// learned step reduces less than the reference runs plain cycles from then on.
//
// Every barrier wait is bounded: after BAR_SPIN_LIMIT polls a CTA raises the
// error word and all CTAs leave the kernel (status CSFF_ERR_TIMEOUT); so is
// every wait for the network's MMAs.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "mg_tiles.cuh"
#include "net_tile.cuh"

namespace csff {
namespace {

constexpr int MAXL = 12;            // levels per instance
constexpr int PT = 2048;            // points per FP64 tile (256 threads x 8)
constexpr long long BAR_SPIN_LIMIT = 1ll << 26;

struct BLevel {
  int m, tc, ntx;                   // interior size, tile size (as fine level), tiles per side
  float2 c;
  tiles::LevelCoef<float> K;        // formed coefficients (separable factors)
  float2 *u, *t, *b;
};

struct BInst {
  int nl, lc, m, n_gauss;
  long long N;
  BLevel L[MAXL];
  tiles::CoarseLevels cl;
  const double2* inv64;             // coarsest inverse, applied in FP64 to the FP32 right-hand side
  double2 c64;
  const double2* q64;
  double2* u64[2];                  // current iterate alternates between these
  double2 *b64, *r64;
  const double2* chi;               // [n_gauss][2][m]
  const double2* uinc;              // [2][m]
  double k2;
  float h2;                         // h^2 of the finest level (the learned step's input scale)
};

struct BState {
  int done, status, cycles, refinements, e, eb, cur, rises, n_hist;
  int n_step;                       // FP32 cycles of the current refinement step
  int lrn, lflags;                  // learned step on; bit 0 a network is set, bit 1 it was switched off
  double lref;                      // reference reduction factor of the learned steps
  double prev, nb, rel;
  double hist[CSFF_MAX_HISTORY];
};

struct BArgs {
  const BInst* inst;
  BState* st;
  int n_inst;
  const int* off_pts;               // [n_inst + 1]
  const int* off_lvl;               // [LC][n_inst + 1] down/up tiles per level
  int LC;
  int inner;                        // cycles per refinement step (at most, when adaptive)
  int adaptive;                     // size each step from the previous step's reduction factor
  double rel_tol;
  int max_cycles;
  double* partials;                 // per FP64 tile
  unsigned* bar;                    // [0] arrivals, [1] generation
  int* err;
  int extra_arrivals;               // test hook: arrivals that never come (0 in use)
  long long spin_limit;             // polls before a barrier wait gives up
  const __nv_bfloat16* net_wb;      // learned smoother's BF16 weights, or null
  double guard;                     // largest reference factor of the learned steps
  const int* off_net;               // [n_inst + 1] network tiles per instance
  int net_off;                      // byte offset of the network's weight region in shared memory
};

__device__ __forceinline__ int find_inst(const int* off, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Grid-wide barrier with a bounded wait.  Returns false if any CTA gave up.
__device__ bool grid_barrier(unsigned* bar, int* err, int extra, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    unsigned gen = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1 + (unsigned)extra) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (*(volatile int*)err) break;
        if (++spins > limit) { atomicExch(err, 1); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = *(volatile int*)err == 0;
  }
  __syncthreads();
  return s_ok;
}

__device__ __forceinline__ bool inst_done(const BState* st, int i) {
  return __ldcg(&st[i].done) != 0;
}

// instance i still runs FP32 cycle c of the current refinement step
__device__ __forceinline__ bool in_cycle(const BState* st, int i, int c) {
  return !inst_done(st, i) && c < __ldcg(&st[i].n_step);
}

// ... and ends it with the learned step
__device__ __forceinline__ bool learned_now(const BState* st, int i, int c) {
  return in_cycle(st, i, c) && __ldcg(&st[i].lrn) != 0;
}

template <typename V>
__device__ __forceinline__ V block_sum(V v, V* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  V s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;
}

__device__ __forceinline__ int frexp_e(double a) {
  int e = 0;
  frexp(a, &e);
  return e;
}

// ---- FP64 point phases --------------------------------------------------------
// rhs: b = k^2 chi u_in, u = 0, r = b; max exponent of |b| into eb
__device__ void ph_rhs(const BInst& I, BState* st, int i, int t) {
  __shared__ int smax;
  if (threadIdx.x == 0) smax = -2000;
  __syncthreads();
  const int m = I.m;
  int mx = -2000;
  for (long long j = (long long)t * PT + threadIdx.x; j < min((long long)(t + 1) * PT, I.N); j += blockDim.x) {
    int ix = (int)(j % m), iy = (int)(j / m);
    double2 cu = make_double2(0, 0);      // chi u_in, axis factors paired first
    for (int g = 0; g < I.n_gauss; ++g) {
      const double2* tb = I.chi + (size_t)g * 2 * m;
      cu = cadd(cu, cmul(cmul(tb[ix], I.uinc[ix]), cmul(tb[m + iy], I.uinc[m + iy])));
    }
    double2 bj = cscale(cu, I.k2);
    I.b64[j] = bj;
    I.r64[j] = bj;
    I.u64[0][j] = make_double2(0, 0);
    double a = fmax(fabs(bj.x), fabs(bj.y));
    int e = (a == 0.0) ? -2000 : (isfinite(a) ? frexp_e(a) : 4000);
    mx = max(mx, e);
  }
  atomicMax(&smax, mx);
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&st[i].eb, smax);
}

// norm partial of r (or b) with the prescale 2^-eb
__device__ void ph_norm(const BInst& I, const BState* st, int i, int t, double* partial, double* shd) {
  const int eb = __ldcg(&st[i].eb);
  const double sc = ldexp(1.0, -min(max(eb, -1000), 1000));
  double acc = 0;
  for (long long j = (long long)t * PT + threadIdx.x; j < min((long long)(t + 1) * PT, I.N); j += blockDim.x) {
    double2 v = __ldcg(I.r64 + j);
    double a = v.x * sc, b = v.y * sc;
    acc = fma(a, a, fma(b, b, acc));
  }
  acc = block_sum(acc, shd);
  if (threadIdx.x == 0) *partial = acc;
}

// r32 = r64 2^-e into the level-0 FP32 right-hand side
__device__ void ph_to32(const BInst& I, const BState* st, int i, int t) {
  const double s = ldexp(1.0, -__ldcg(&st[i].e));
  for (long long j = (long long)t * PT + threadIdx.x; j < min((long long)(t + 1) * PT, I.N); j += blockDim.x) {
    double2 r = __ldcg(I.r64 + j);
    I.L[0].b[j] = make_float2((float)(r.x * s), (float)(r.y * s));
  }
}

// u_new = u + 2^e e32; r = b - A u_new (neighbours formed on the fly from the
// old iterate, which stays untouched); norm partial of r
__device__ void ph_update(const BInst& I, const BState* st, int i, int t, double* partial, double* shd) {
  const int cur = __ldcg(&st[i].cur);
  const double2* uo = I.u64[cur];
  double2* un = I.u64[cur ^ 1];
  const float2* e32 = I.L[0].u;
  const double s = ldexp(1.0, __ldcg(&st[i].e));
  const int eb = __ldcg(&st[i].eb);
  const double sc = ldexp(1.0, -min(max(eb, -1000), 1000));
  const int m = I.m;
  auto v_at = [&](long long j) {
    double2 u = __ldcg(uo + j);
    float2 e = __ldcg(e32 + j);
    return make_double2(fma((double)e.x, s, u.x), fma((double)e.y, s, u.y));
  };
  double acc = 0;
  for (long long j = (long long)t * PT + threadIdx.x; j < min((long long)(t + 1) * PT, I.N); j += blockDim.x) {
    int ix = (int)(j % m), iy = (int)(j / m);
    double2 vj = v_at(j);
    double2 nb = make_double2(0, 0);
    if (ix > 0) nb = cadd(nb, v_at(j - 1));
    if (ix < m - 1) nb = cadd(nb, v_at(j + 1));
    if (iy > 0) nb = cadd(nb, v_at(j - m));
    if (iy < m - 1) nb = cadd(nb, v_at(j + m));
    double2 tt = csub(cscale(vj, 4.0), nb);
    double2 au = csub(cmul(I.c64, tt), cmul(I.q64[j], vj));
    double2 r = csub(__ldcg(I.b64 + j), au);
    un[j] = vj;
    I.r64[j] = r;
    double a = r.x * sc, b = r.y * sc;
    acc = fma(a, a, fma(b, b, acc));
  }
  acc = block_sum(acc, shd);
  if (threadIdx.x == 0) *partial = acc;
}

// per-instance reduction of the norm partials and the convergence decision
__device__ void ph_finish(const BArgs& A, int i, bool initial, double* shd) {
  const int p0 = A.off_pts[i], p1 = A.off_pts[i + 1];
  double acc = 0;
  for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) acc += __ldcg(A.partials + p);
  acc = block_sum(acc, shd);
  if (threadIdx.x != 0) return;
  BState& S = A.st[i];
  const int eb = S.eb;
  const double nrm = sqrt(acc) * ldexp(1.0, min(max(eb, -1000), 1000));
  if (initial) {
    S.nb = nrm;
    S.hist[0] = 1.0;
    S.n_hist = 1;
    S.prev = 1.0;
    S.rel = 1.0;
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      S.done = 1;
      S.status = (nrm == 0.0) ? CSFF_OK : CSFF_ERR_NONFINITE;
      S.rel = 0.0;
    }
    S.e = frexp_e(nrm);
    S.n_step = A.inner;
    S.lrn = 0;
    S.lflags = A.net_wb ? 1 : 0;
    S.lref = A.guard;
    return;
  }
  const double rel = nrm / S.nb;
  const double rel_before = S.rel;
  const int ran = S.n_step;
  S.cycles += ran;
  S.refinements += 1;
  S.rel = rel;
  if (S.n_hist < CSFF_MAX_HISTORY) S.hist[S.n_hist++] = rel;
  S.cur ^= 1;
  S.e = frexp_e(nrm);
  int status = -1;
  if (!isfinite(rel)) status = CSFF_ERR_NONFINITE;
  else if (rel <= A.rel_tol) status = CSFF_OK;
  else {
    S.rises = rel > S.prev ? S.rises + 1 : 0;
    S.prev = rel;
    if (S.rises >= 3) status = CSFF_ERR_DIVERGED;
    else if (S.cycles >= A.max_cycles) status = CSFF_ERR_NOT_CONVERGED;
  }
  if (A.net_wb) {
    // the learned step: off for the first two refinement steps, the second's
    // factor is the reference; a learned step that reduces less turns it off
    // (factors of steps of inner cycles: the adaptive schedule's steps differ)
    const double factor = ran == A.inner ? rel / rel_before : pow(rel / rel_before, (double)A.inner / ran);
    if (S.refinements <= 2) {
      if (S.refinements == 2) {
        S.lref = fmin(factor, A.guard);
        S.lrn = 1;
      }
    } else if (S.lrn && factor > S.lref) {
      S.lrn = 0;
      S.lflags |= 2;
    }
  }
  if (status >= 0) {
    S.status = status;
    S.done = 1;
  } else if (A.adaptive) {
    S.n_step = refinement_cycles(rel_before, rel, ran, A.rel_tol, A.inner);
  }
}

// r = b - A u on the finest level in FP32 (the learned step's input), with the
// coefficients formed from the separable factors as in the tiles:
// A u = d u - c sum_nbr u, d = 4c - k^2 - sum_g X_g Y_g
__device__ void ph_resid0(const BInst& I, int t) {
  const BLevel& F = I.L[0];
  const int m = F.m;
  const long long N = (long long)m * m;
  const float2 c = F.c;
  const float2 D0 = make_float2(__fmaf_rn(4.f, c.x, -F.K.k2), __fmul_rn(4.f, c.y));
  for (int k = 0; k < PT / 256; ++k) {
    const long long j = (long long)t * PT + k * 256 + threadIdx.x;
    if (j >= N) return;
    const int iy = (int)(j / m), ix = (int)(j - (long long)iy * m);
    float2 d = D0;
    for (int g = 0; g < F.K.ng; ++g) {
      const float2* f = F.K.fac + (size_t)g * 2 * m;
      d = tiles::xfms(d, f[ix], f[m + iy]);
    }
    const float2 uj = F.u[j];
    float2 sn = make_float2(0.f, 0.f);
    if (ix > 0) sn = tiles::xadd(sn, F.u[j - 1]);
    if (ix < m - 1) sn = tiles::xadd(sn, F.u[j + 1]);
    if (iy > 0) sn = tiles::xadd(sn, F.u[j - m]);
    if (iy < m - 1) sn = tiles::xadd(sn, F.u[j + m]);
    F.t[j] = tiles::xfma(tiles::xfms(F.b[j], d, uj), c, sn);          // b - d u + c s
  }
}

// the first network work item at or after `from` (in steps of the grid) whose
// instance takes the learned step in cycle c, or the total
__device__ int next_net_item(const BArgs& A, int c, int from) {
  const int n = A.n_inst, total = A.off_net[n];
  for (int it = from; it < total; it += gridDim.x)
    if (learned_now(A.st, find_inst(A.off_net, n, it), c)) return it;
  return total;
}

// network work item it: an output tile of its instance's finest level, input
// r in the level's t buffer, output u
__device__ nettile::Tile net_item(const BArgs& A, int it, float* scale) {
  const int i = find_inst(A.off_net, A.n_inst, it);
  const BInst& I = A.inst[i];
  const int t = it - A.off_net[i], tiles_x = (I.m + nettile::TW - 1) / nettile::TW;
  *scale = I.h2;
  return nettile::Tile{I.L[0].t, I.L[0].u, I.m, I.m, (t % tiles_x) * nettile::TW - 3,
                       (t / tiles_x) * nettile::TH - 3};
}

// the network phase of cycle c: every output tile of every instance that takes
// the learned step, u += N(h^2 r); the next tile's input is loaded while the
// current tile's MMAs run.  Kept out of line: the kernel body stays small
// enough for every host build of the compiler.
__device__ __noinline__ bool ph_net(const BArgs& A, int c, nettile::mmat::Ctx& nc) {
  const int total = A.off_net[A.n_inst];
  int it = next_net_item(A, c, blockIdx.x);
  if (it >= total) return true;
  for (int i = threadIdx.x; i < nettile::PLANES_BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(nc.planes)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  float2 xr[nettile::SPT];
  float scale = 1.f, next_scale = 1.f;
  nettile::Tile cur = net_item(A, it, &scale);
  nettile::load_x(cur, xr);
  while (it < total) {
    const int nxt = next_net_item(A, c, it + gridDim.x);
    const nettile::Tile next = net_item(A, nxt < total ? nxt : it, &next_scale);
    if (!nettile::mmat::run_tile(nc, cur, xr, scale, 1, nxt < total ? &next : nullptr)) return false;
    cur = next;
    scale = next_scale;
    it = nxt;
  }
  return true;
}

// ---- FP32 V-cycle phases --------------------------------------------------------
__device__ void ph_down(const BInst& I, int l, int t, bool zero_init, unsigned char* smem) {
  const BLevel& F = I.L[l];
  const BLevel& C = I.L[l + 1];
  const int tx = t % F.ntx, ty = t / F.ntx;
  const float2* in = (l == 0) ? F.u : nullptr;
  bool zi = zero_init || l > 0;
  const bool g1 = F.K.ng == 1;
  if (F.tc == 16) {
    if (g1) tiles::down_tile<float, 16, true, true>(tx * 16, ty * 16, in, zi, F.b, F.K, F.c, F.m, C.m, F.t, C.b, smem);
    else tiles::down_tile<float, 16, true, false>(tx * 16, ty * 16, in, zi, F.b, F.K, F.c, F.m, C.m, F.t, C.b, smem);
  } else {
    if (g1) tiles::down_tile<float, 8, true, true>(tx * 8, ty * 8, in, zi, F.b, F.K, F.c, F.m, C.m, F.t, C.b, smem);
    else tiles::down_tile<float, 8, true, false>(tx * 8, ty * 8, in, zi, F.b, F.K, F.c, F.m, C.m, F.t, C.b, smem);
  }
}

__device__ void ph_up(const BInst& I, int l, int t, unsigned char* smem) {
  const BLevel& F = I.L[l];
  const BLevel& C = I.L[l + 1];
  const int tx = t % F.ntx, ty = t / F.ntx;
  const bool g1 = F.K.ng == 1;
  if (F.tc == 16) {
    if (g1) tiles::up_tile<float, 16, true, true>(tx * 16, ty * 16, F.t, C.u, F.b, F.K, F.c, F.m, C.m, F.u, smem);
    else tiles::up_tile<float, 16, true, false>(tx * 16, ty * 16, F.t, C.u, F.b, F.K, F.c, F.m, C.m, F.u, smem);
  } else {
    if (g1) tiles::up_tile<float, 8, true, true>(tx * 8, ty * 8, F.t, C.u, F.b, F.K, F.c, F.m, C.m, F.u, smem);
    else tiles::up_tile<float, 8, true, false>(tx * 8, ty * 8, F.t, C.u, F.b, F.K, F.c, F.m, C.m, F.u, smem);
  }
}

template <bool LEARNED>
__device__ __forceinline__ void batch_body(const BArgs& A, unsigned char* smem, double* shd, nettile::mmat::Ctx& nc) {
  const int n = A.n_inst;
  const int npts = A.off_pts[n];
  // ---- initial residual r = b (u = 0) and its norm
  for (int it = blockIdx.x; it < npts; it += gridDim.x) {
    int i = find_inst(A.off_pts, n, it);
    ph_rhs(A.inst[i], A.st, i, it - A.off_pts[i]);
  }
  if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
  for (int it = blockIdx.x; it < npts; it += gridDim.x) {
    int i = find_inst(A.off_pts, n, it);
    ph_norm(A.inst[i], A.st, i, it - A.off_pts[i], A.partials + it, shd);
  }
  if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
  for (int i = blockIdx.x; i < n; i += gridDim.x) ph_finish(A, i, true, shd);
  if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;

  for (;;) {
    bool any = false;
    for (int i = 0; i < n; ++i) any |= !inst_done(A.st, i);
    if (!any) break;
    for (int it = blockIdx.x; it < npts; it += gridDim.x) {
      int i = find_inst(A.off_pts, n, it);
      if (!inst_done(A.st, i)) ph_to32(A.inst[i], A.st, i, it - A.off_pts[i]);
    }
    if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
    for (int c = 0; c < A.inner; ++c) {
      // instances whose step is shorter sit out its remaining cycles (every
      // CTA reads the same state, so all leave the loop together)
      bool busy = false;
      for (int i = 0; i < n; ++i) busy |= in_cycle(A.st, i, c);
      if (!busy) break;
      for (int l = 0; l < A.LC; ++l) {
        const int* off = A.off_lvl + (size_t)l * (n + 1);
        for (int it = blockIdx.x; it < off[n]; it += gridDim.x) {
          int i = find_inst(off, n, it);
          if (in_cycle(A.st, i, c)) ph_down(A.inst[i], l, it - off[i], c == 0, smem);
        }
        if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
      }
      for (int i = blockIdx.x; i < n; i += gridDim.x) {
        if (!in_cycle(A.st, i, c)) continue;
        const BInst& I = A.inst[i];
        tiles::coarse_levels_block<float, 2, true, double>(I.cl, I.L[I.lc].b, I.L[I.lc].u, I.inv64, smem);
      }
      if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
      for (int l = A.LC - 1; l >= 0; --l) {
        const int* off = A.off_lvl + (size_t)l * (n + 1);
        for (int it = blockIdx.x; it < off[n]; it += gridDim.x) {
          int i = find_inst(off, n, it);
          if (in_cycle(A.st, i, c)) ph_up(A.inst[i], l, it - off[i], smem);
        }
        if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
      }
      if constexpr (LEARNED) {
        bool any = false;
        for (int i = 0; i < n; ++i) any |= learned_now(A.st, i, c);
        if (any) {
          for (int it = blockIdx.x; it < npts; it += gridDim.x) {
            int i = find_inst(A.off_pts, n, it);
            if (learned_now(A.st, i, c)) ph_resid0(A.inst[i], it - A.off_pts[i]);
          }
          if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
          if (!ph_net(A, c, nc)) return;
          if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
        }
      }
    }
    for (int it = blockIdx.x; it < npts; it += gridDim.x) {
      int i = find_inst(A.off_pts, n, it);
      if (!inst_done(A.st, i)) ph_update(A.inst[i], A.st, i, it - A.off_pts[i], A.partials + it, shd);
    }
    if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
    for (int i = blockIdx.x; i < n; i += gridDim.x)
      if (!inst_done(A.st, i)) ph_finish(A, i, false, shd);
    if (!grid_barrier(A.bar, A.err, A.extra_arrivals, A.spin_limit)) return;
  }
}

// at most 85 registers a thread, so that three CTAs fit on an SM (the
// autotuner picks between one and the occupancy maximum).  LEARNED: the
// learned step ends every cycle; each CTA holds the network's weight operands
// for the whole launch, and the activation planes share the tiles' shared
// memory.  The network runs on the warp-level MMA instructions: the occupancy
// calculation, which bounds a cooperative launch, admits one CTA per SM for any
// kernel with tensor-memory instructions.
template <bool LEARNED>
__global__ void __launch_bounds__(256, 3) k_batch_solve(BArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double shd[8];
  nettile::mmat::Ctx nc;
  if constexpr (LEARNED) nettile::mmat::setup(nc, smem, smem + A.net_off, A.net_wb);
  batch_body<LEARNED>(A, smem, shd, nc);
}

__global__ void k_batch_init(BState* st, int n, unsigned* bar, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) { bar[0] = 0; bar[1] = 0; *err = 0; }
  if (i >= n) return;
  BState& S = st[i];
  S.done = 0; S.status = 0; S.cycles = 0; S.refinements = 0; S.e = 0; S.eb = -2000; S.cur = 0;
  S.rises = 0; S.n_hist = 0; S.prev = 1.0; S.nb = 0.0; S.rel = 1.0; S.n_step = 1;
  S.lrn = 0; S.lflags = 0; S.lref = 1.0;
}

size_t batch_smem(const std::vector<csff_plan*>& plans) {
  int ng = 0;
  for (csff_plan* P : plans) ng = std::max(ng, P->prob.n_gauss);
  size_t s = std::max(tiles::down_smem_elems<16>(ng, false), tiles::up_smem_elems<16>(ng, false));
  for (csff_plan* P : plans) {
    int lc = P->fused_lc;
    s = std::max(s, tiles::coarse_levels_elems(P->lv, lc));
  }
  return s * sizeof(float2);
}

}  // namespace
}  // namespace csff

using csff::BArgs;
using csff::BInst;
using csff::BState;

struct csff_batch {
  int n = 0;
  int LC = 0;
  std::vector<csff_plan*> plans;
  cudaStream_t stream = nullptr;
  csff_opts opts{};
  BInst* d_inst = nullptr;
  BState* d_state = nullptr;
  BState* h_state = nullptr;      // pinned
  int* d_off = nullptr;           // off_pts then off_lvl
  double* d_partials = nullptr;
  unsigned* d_bar = nullptr;
  int* d_err = nullptr;
  double2* h_uinc = nullptr;      // pinned staging of incident tables
  int h_err = 0;
  int* h_err_p = nullptr;         // pinned error word mirror
  cudaStream_t gstream = nullptr; // capture/replay stream
  uint64_t gkernels = 0;
  cudaEvent_t gev = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = true;
  int dbg_extra = 0;              // csff_batch_debug_barrier
  long long dbg_spin = 0;
  size_t smem = 0;
  int tc_big = 16;                // tuned: tile size of levels with >= 64 coarse points per side
  int ctas_per_sm = 0;            // tuned: 0 = occupancy maximum
  int grid = 0;
  bool tuned = false;
  std::vector<int> off_host;
  csff_net* net = nullptr;        // learned smoother (csff_batch_set_learned), not owned
  double guard = 0.5;
  size_t smem_tiles = 0;          // shared memory of the tile phases
  int net_off = 0;
};

namespace {

#define BK(call, what)                                                   \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return csff::cuda_fail(e_, what);             \
  } while (0)

csff_status binvalid(const char* s) {
  csff::set_error(s);
  return CSFF_ERR_INVALID_ARG;
}

// the persistent kernel of the batch's form
const void* batch_kernel(const csff_batch* B) {
  return B->net ? (const void*)csff::k_batch_solve<true> : (const void*)csff::k_batch_solve<false>;
}

// device descriptors of every instance for the current tile choice
csff_status upload_descriptors(csff_batch* B) {
  const int n = B->n;
  std::vector<BInst> hi(n);
  int LC = 0;
  for (int i = 0; i < n; ++i) LC = std::max(LC, B->plans[i]->fused_lc);
  B->LC = LC;
  std::vector<int> off_pts(n + 1, 0), off_lvl((size_t)LC * (n + 1), 0), off_net(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    csff_plan* P = B->plans[i];
    BInst& I = hi[i];
    std::memset(&I, 0, sizeof(I));
    I.nl = (int)P->lv.size();
    I.lc = P->fused_lc;
    I.m = P->lv[0].m;
    I.N = P->lv[0].N;
    I.n_gauss = P->prob.n_gauss;
    for (int l = 0; l < I.nl && l < csff::MAXL; ++l) {
      csff::Level& L = P->lv[l];
      csff::BLevel& b = I.L[l];
      b.m = L.m;
      int mc = (l + 1 < I.nl) ? P->lv[l + 1].m : 1;
      b.tc = (mc >= 64) ? B->tc_big : 8;
      b.ntx = (mc + b.tc - 1) / b.tc;
      b.c = make_float2((float)L.c.x, (float)L.c.y);
      b.K = csff::tiles::LevelCoef<float>{};
      b.K.fac = L.fac32;
      b.K.ng = L.ng;
      b.K.k2 = (float)L.k2;
      b.u = L.u32;
      b.t = L.t32;
      b.b = L.b32;
    }
    I.cl.nl = I.nl - I.lc;
    for (int l = 0; l < I.cl.nl; ++l) {
      csff::Level& L = P->lv[I.lc + l];
      I.cl.m[l] = L.m;
      I.cl.q[l] = L.q32;
      I.cl.dinv[l] = L.dinv32;
      I.cl.c[l] = L.c;
      I.cl.c32[l] = make_float2((float)L.c.x, (float)L.c.y);
    }
    I.inv64 = P->coarse_inv;
    I.c64 = P->lv[0].c;
    I.q64 = P->lv[0].q64;
    I.u64[0] = P->lv[0].u64;
    I.u64[1] = P->lv[0].t64;
    I.b64 = P->lv[0].b64;
    I.r64 = P->lv[0].r64;
    I.chi = P->chi_tab[0];
    I.uinc = P->uinc_tab;
    I.k2 = P->prob.k * P->prob.k;
    I.h2 = (float)(P->lv[0].h * P->lv[0].h);
    off_pts[i + 1] = off_pts[i] + (int)((I.N + csff::PT - 1) / csff::PT);
    off_net[i + 1] = off_net[i] + ((I.m + csff::nettile::TW - 1) / csff::nettile::TW) *
                                      ((I.m + csff::nettile::TH - 1) / csff::nettile::TH);
    for (int l = 0; l < LC; ++l) {
      int t = (l < I.lc) ? I.L[l].ntx * I.L[l].ntx : 0;
      off_lvl[(size_t)l * (n + 1) + i + 1] = off_lvl[(size_t)l * (n + 1) + i] + t;
    }
  }
  B->off_host = off_pts;
  B->off_host.insert(B->off_host.end(), off_lvl.begin(), off_lvl.end());
  B->off_host.insert(B->off_host.end(), off_net.begin(), off_net.end());
  BK(cudaMemcpy(B->d_inst, hi.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice), "upload batch descriptors");
  if (B->d_off) cudaFree(B->d_off);
  BK(cudaMalloc((void**)&B->d_off, sizeof(int) * B->off_host.size()), "batch tables");
  BK(cudaMemcpy(B->d_off, B->off_host.data(), sizeof(int) * B->off_host.size(), cudaMemcpyHostToDevice),
     "upload batch tables");
  if (B->d_partials) cudaFree(B->d_partials);
  BK(cudaMalloc((void**)&B->d_partials, sizeof(double) * std::max(1, off_pts[n])), "batch partials");
  return CSFF_OK;
}

csff_status launch_batch(csff_batch* B, cudaStream_t s) {
  const int n = B->n;
  int dev = 0, sms = 0, occ = 0;
  BK(cudaGetDevice(&dev), "device");
  BK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  const void* kern = batch_kernel(B);
  BK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem), "batch smem");
  BK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, B->smem), "occupancy");
  if (occ < 1) return binvalid("batch kernel does not fit on an SM");
  int per = B->ctas_per_sm > 0 ? std::min(B->ctas_per_sm, occ) : occ;
  B->grid = per * sms;
  csff::k_batch_init<<<(n + 255) / 256, 256, 0, s>>>(B->d_state, n, B->d_bar, B->d_err);
  csff::count_launch();
  BArgs A;
  A.inst = B->d_inst;
  A.st = B->d_state;
  A.n_inst = n;
  A.off_pts = B->d_off;
  A.off_lvl = B->d_off + (n + 1);
  A.LC = B->LC;
  A.inner = B->opts.inner_cycles > 0 ? B->opts.inner_cycles : 1;
  A.adaptive = B->opts.adaptive_inner != 0 ? 1 : 0;
  A.rel_tol = B->opts.rel_tol;
  A.max_cycles = B->opts.max_cycles;
  A.partials = B->d_partials;
  A.bar = B->d_bar;
  A.err = B->d_err;
  A.extra_arrivals = B->dbg_extra;
  A.spin_limit = B->dbg_spin > 0 ? B->dbg_spin : csff::BAR_SPIN_LIMIT;
  A.net_wb = B->net ? (const __nv_bfloat16*)csff::net_weights_bf16(B->net) : nullptr;
  A.guard = B->guard;
  A.off_net = B->d_off + (size_t)(n + 1) * (1 + B->LC);
  A.net_off = B->net_off;
  void* args[] = {&A};
  {
    csff::ProfScope ps(csff::PF_MG32, s, 0, 0);
    BK(cudaLaunchCooperativeKernel(kern, dim3(B->grid), dim3(256), args, B->smem, s), "cooperative batch launch");
  }
  csff::count_launch();
  return CSFF_OK;
}

// incident-wave tables of every instance into the pinned staging buffer
void fill_incident(csff_batch* B, const double* eta) {
  size_t off = 0;
  for (int i = 0; i < B->n; ++i) {
    csff_plan* P = B->plans[i];
    const int m = P->lv[0].m;
    const std::complex<double> ik(0.0, P->prob.k), rot = std::polar(1.0, P->prob.gamma);
    for (int c = 0; c < 2; ++c)
      for (int j = 0; j < m; ++j) {
        double x = P->prob.box_lo + (j + 1) * P->lv[0].h;
        std::complex<double> v = std::exp(ik * eta[2 * i + c] * x * rot);
        B->h_uinc[off + (size_t)c * m + j] = make_double2(v.real(), v.imag());
      }
    off += 2 * (size_t)m;
  }
}

// the device work of one batched solve: staged uploads, state init, the
// persistent kernel, state readback (capturable: pinned buffers only)
csff_status enqueue_solve(csff_batch* B, cudaStream_t s) {
  size_t off = 0;
  for (int i = 0; i < B->n; ++i) {
    csff_plan* P = B->plans[i];
    const int m = P->lv[0].m;
    BK(cudaMemcpyAsync(P->uinc_tab, B->h_uinc + off, sizeof(double2) * 2 * m, cudaMemcpyHostToDevice, s),
       "upload incident tables");
    off += 2 * (size_t)m;
  }
  csff_status st = launch_batch(B, s);
  if (st != CSFF_OK) return st;
  BK(cudaMemcpyAsync(B->h_state, B->d_state, sizeof(BState) * B->n, cudaMemcpyDeviceToHost, s), "states");
  BK(cudaMemcpyAsync(B->h_err_p, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "error word");
  return CSFF_OK;
}

// run one solve: replay the captured graph (capture on first use); fall back
// to direct launches if the capture is refused
csff_status run_solve(csff_batch* B) {
  if (csff::prof_mask() != 0) B->graph_ok = false;
  BK(cudaEventRecord(B->gev, B->stream), "event");
  BK(cudaStreamWaitEvent(B->gstream, B->gev, 0), "wait");
  if (B->graph_ok && !B->gexec) {
    const uint64_t before = csff::g_launches.load();
    if (cudaStreamBeginCapture(B->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      csff::g_capturing = true;
      csff_status st = enqueue_solve(B, B->gstream);
      csff::g_capturing = false;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(B->gstream, &g);
      if (st == CSFF_OK && e == cudaSuccess && g && cudaGraphInstantiate(&B->gexec, g, 0) == cudaSuccess) {
        B->gkernels = csff::g_launches.load() - before;
      } else {
        B->gexec = nullptr;
        B->graph_ok = false;
      }
      csff::g_launches.store(before);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();   // a refused capture leaves no sticky error
    } else {
      cudaGetLastError();
      B->graph_ok = false;
    }
  }
  if (B->gexec) {
    BK(cudaGraphLaunch(B->gexec, B->gstream), "graph launch");
    csff::count_launch((int)B->gkernels);
  } else {
    csff_status st = enqueue_solve(B, B->gstream);
    if (st != CSFF_OK) return st;
  }
  BK(cudaStreamSynchronize(B->gstream), "batch sync");
  return CSFF_OK;
}

csff_status collect(csff_batch* B, csff_info* infos, int* worst) {
  const int err = *B->h_err_p;
  *worst = CSFF_OK;
  if (err) {
    csff::set_error("batch kernel: a grid barrier or tensor-core wait ran out");
    *worst = CSFF_ERR_TIMEOUT;
  }
  for (int i = 0; i < B->n; ++i) {
    const BState& S = B->h_state[i];
    int st = err ? CSFF_ERR_TIMEOUT : (S.done ? S.status : CSFF_ERR_NOT_CONVERGED);
    if (st != CSFF_OK && *worst == CSFF_OK) *worst = st;
    if (infos) {
      csff_info& in = infos[i];
      std::memset(&in, 0, sizeof(in));
      in.status = st;
      in.cycles = S.cycles;
      in.refinements = S.refinements;
      in.rel_res = S.rel;
      in.conv_factor = S.cycles > 0 ? std::pow(S.rel, 1.0 / S.cycles) : 0.0;
      in.n_hist = S.n_hist;
      in.flags = S.lflags;
      for (int h = 0; h < S.n_hist && h < CSFF_MAX_HISTORY; ++h) in.history[h] = S.hist[h];
    }
  }
  return CSFF_OK;
}

}  // namespace

extern "C" {

void csff_batch_destroy(csff_batch* B) {
  if (!B) return;
  for (csff_plan* P : B->plans) csff_plan_destroy(P);
  for (void* p : {(void*)B->d_inst, (void*)B->d_state, (void*)B->d_off, (void*)B->d_partials, (void*)B->d_bar,
                  (void*)B->d_err})
    if (p) cudaFree(p);
  if (B->h_state) cudaFreeHost(B->h_state);
  if (B->h_uinc) cudaFreeHost(B->h_uinc);
  if (B->h_err_p) cudaFreeHost(B->h_err_p);
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->gstream) cudaStreamDestroy(B->gstream);
  if (B->gev) cudaEventDestroy(B->gev);
  delete B;
}

csff_status csff_batch_create(int n_inst, const csff_problem* probs, const csff_opts* opts, void* stream,
                              csff_batch** out) {
  if (!out) return binvalid("out is NULL");
  *out = nullptr;
  if (n_inst < 1 || n_inst > 4096 || !probs || !opts) return binvalid("need 1..4096 problems and options");
  if (opts->smoother != CSFF_SMOOTHER_RBGS || opts->nu1 != 1 || opts->nu2 != 1 || opts->precision != CSFF_PREC_MIXED) {
    csff::set_error("batched solve: needs red-black GS V(1,1) with mixed precision");
    return CSFF_ERR_UNSUPPORTED;
  }
  csff_batch* B = new csff_batch();
  B->n = n_inst;
  B->opts = *opts;
  B->stream = (cudaStream_t)stream;
  auto fail = [&](csff_status s) {
    csff_batch_destroy(B);
    return s;
  };
  size_t uinc_total = 0;
  for (int i = 0; i < n_inst; ++i) {
    if (probs[i].dim != 2) return fail(binvalid("batched solve: 2D problems only"));
    csff_plan* P = nullptr;
    csff_status s = csff_plan_create(&probs[i], opts, stream, &P);
    if (s != CSFF_OK) return fail(s);
    B->plans.push_back(P);
    if (P->fused_lc < 1 || (int)P->lv.size() > csff::MAXL) {
      csff::set_error("batched solve: each grid needs n >= 65 and at most 12 levels");
      return fail(CSFF_ERR_UNSUPPORTED);
    }
    uinc_total += 2 * (size_t)P->lv[0].m;
  }
  cudaError_t e;
  if ((e = cudaMalloc((void**)&B->d_inst, sizeof(BInst) * n_inst)) != cudaSuccess ||
      (e = cudaMalloc((void**)&B->d_state, sizeof(BState) * n_inst)) != cudaSuccess ||
      (e = cudaMalloc((void**)&B->d_bar, 2 * sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMalloc((void**)&B->d_err, sizeof(int))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&B->h_state, sizeof(BState) * n_inst)) != cudaSuccess ||
      (e = cudaMallocHost((void**)&B->h_uinc, sizeof(double2) * uinc_total)) != cudaSuccess ||
      (e = cudaMallocHost((void**)&B->h_err_p, sizeof(int))) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&B->gstream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&B->gev, cudaEventDisableTiming)) != cudaSuccess)
    return fail(csff::cuda_fail(e, "batch allocation"));
  B->smem = B->smem_tiles = csff::batch_smem(B->plans);
  if (B->smem > 227 * 1024) return fail(binvalid("batched solve: coarse levels exceed shared memory"));
  csff_status s = upload_descriptors(B);
  if (s != CSFF_OK) return fail(s);
  *out = B;
  return CSFF_OK;
}

csff_status csff_batch_solve(csff_batch* B, const double* eta, csff_info* infos) {
  if (!B || !eta) return binvalid("NULL argument");
  fill_incident(B, eta);
  csff_status s = run_solve(B);
  if (s != CSFF_OK) return s;
  int worst = CSFF_OK;
  if ((s = collect(B, infos, &worst)) != CSFF_OK) return s;
  return (csff_status)worst;
}

csff_status csff_batch_solution(const csff_batch* B, int i, const void** u_dev) {
  if (!B || !u_dev || i < 0 || i >= B->n) return binvalid("bad instance index");
  const csff_plan* P = B->plans[i];
  // the iterate alternates between two buffers; cur says which holds it
  *u_dev = B->h_state[i].cur ? (const void*)P->lv[0].t64 : (const void*)P->lv[0].u64;
  return CSFF_OK;
}

csff_status csff_batch_copy_solution(const csff_batch* B, int i, void* u_out_dev) {
  const void* u = nullptr;
  csff_status s = csff_batch_solution(B, i, &u);
  if (s != CSFF_OK) return s;
  if (!u_out_dev) return binvalid("NULL output");
  const csff_plan* P = B->plans[i];
  BK(cudaMemcpyAsync(u_out_dev, u, sizeof(double2) * (size_t)P->lv[0].N, cudaMemcpyDeviceToDevice, B->stream),
     "copy solution");
  BK(cudaStreamSynchronize(B->stream), "sync");
  return CSFF_OK;
}

csff_status csff_batch_far_field(csff_batch* B, const double* eta, const int* n_ang, const double* const* alpha,
                                 void* const* F_dev, int32_t* const* F_exp_dev) {
  if (!B || !eta || !n_ang || !alpha || !F_dev) return binvalid("NULL argument");
  for (int i = 0; i < B->n; ++i) {
    const void* u = nullptr;
    csff_status s = csff_batch_solution(B, i, &u);
    if (s != CSFF_OK) return s;
    csff_plan* P = B->plans[i];
    P->stream = B->stream;
    s = csff::far_field_one(P, eta + 2 * i, (const double2*)u, n_ang[i], alpha[i], (double2*)F_dev[i],
                            F_exp_dev ? F_exp_dev[i] : nullptr, nullptr);
    if (s != CSFF_OK) return s;
  }
  return CSFF_OK;
}

csff_status csff_batch_debug_barrier(csff_batch* B, int extra_arrivals, long long spin_limit) {
  if (!B || extra_arrivals < 0 || extra_arrivals > 1 || spin_limit < 0) return binvalid("bad debug settings");
  B->dbg_extra = extra_arrivals;
  B->dbg_spin = spin_limit;
  if (B->gexec) { cudaGraphExecDestroy(B->gexec); B->gexec = nullptr; }   // parameters are baked into the graph
  return CSFF_OK;
}

csff_status csff_batch_set_learned(csff_batch* B, csff_net* net, double guard) {
  if (!B) return binvalid("NULL batch");
  if (net && !(guard > 0.0)) return binvalid("guard must be positive");
  if (net && csff::net_dim(net) != 2) return binvalid("batched solve: needs a 2D network");
  B->net = net;
  B->guard = guard;
  if (net) {
    // the network's activation planes share the tiles' shared memory; its
    // weight operands, mbarrier and tensor-memory slot follow
    const size_t planes = std::max<size_t>((B->smem_tiles + 127) / 128 * 128, csff::nettile::PLANES_BYTES);
    B->net_off = (int)planes;
    B->smem = planes + csff::nettile::WREG_BYTES;
    if (B->smem > 227 * 1024) {
      B->net = nullptr;
      B->smem = B->smem_tiles;
      return binvalid("batched solve: the learned step does not fit in shared memory");
    }
  } else {
    B->net_off = 0;
    B->smem = B->smem_tiles;
  }
  if (B->gexec) { cudaGraphExecDestroy(B->gexec); B->gexec = nullptr; }   // parameters are baked into the graph
  return CSFF_OK;
}

csff_status csff_batch_set_tiles(csff_batch* B, int tc_big, int ctas_per_sm) {
  if (!B) return binvalid("NULL batch");
  if (tc_big != 8 && tc_big != 16) return binvalid("tile size must be 8 or 16 coarse points");
  if (ctas_per_sm < 0) return binvalid("ctas_per_sm must be >= 0");
  B->tc_big = tc_big;
  B->ctas_per_sm = ctas_per_sm;
  if (B->gexec) { cudaGraphExecDestroy(B->gexec); B->gexec = nullptr; }   // parameters are baked into the graph
  return upload_descriptors(B);
}

csff_status csff_batch_autotune(csff_batch* B, const double* eta, int* tc_big_out, int* ctas_per_sm_out) {
  if (!B || !eta) return binvalid("NULL argument");
  int dev = 0, sms = 0, occ = 0;
  BK(cudaGetDevice(&dev), "device");
  BK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  const void* kern = batch_kernel(B);
  BK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem), "batch smem");
  BK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, B->smem), "occupancy");
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0), "event");
  BK(cudaEventCreate(&e1), "event");
  float best = 1e30f;
  int best_tc = B->tc_big, best_per = B->ctas_per_sm;
  fill_incident(B, eta);
  if (B->gexec) { cudaGraphExecDestroy(B->gexec); B->gexec = nullptr; }
  csff_status s = CSFF_OK;
  for (int tc : {16, 8}) {
    B->tc_big = tc;
    if (s == CSFF_OK) s = upload_descriptors(B);
    for (int per = 1; per <= occ && s == CSFF_OK; ++per) {
      B->ctas_per_sm = per;
      float ms = 0;
      for (int rep = 0; rep < 2 && s == CSFF_OK; ++rep) {   // first run warms up
        cudaEventRecord(e0, B->gstream);
        s = enqueue_solve(B, B->gstream);
        cudaEventRecord(e1, B->gstream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) s = csff::cuda_fail(e, "autotune");
        cudaEventElapsedTime(&ms, e0, e1);
      }
      int err = *B->h_err_p;
      if (s == CSFF_OK && !err && ms < best) {
        best = ms;
        best_tc = tc;
        best_per = per;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != CSFF_OK) return s;
  B->tc_big = best_tc;
  B->ctas_per_sm = best_per;
  B->tuned = true;
  csff_status u = upload_descriptors(B);
  if (u != CSFF_OK) return u;
  if (tc_big_out) *tc_big_out = best_tc;
  if (ctas_per_sm_out) *ctas_per_sm_out = best_per;
  return CSFF_OK;
}

}  // extern "C"
