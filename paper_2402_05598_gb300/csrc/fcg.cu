// Flexible conjugate gradients (Algorithm 1, Section 2.3) for a batch of independent
// instances, FP64 throughout the Krylov loop.
//
// Iteration i of instance b:
//   w_i = B(r_i)                                  (preconditioner, another translation unit)
//   m_i = min(i, max(1, i mod (m_max+1)))
//   beta_k = (w_i, s_k) / (p_k, s_k),   k = i-m_i .. i-1   (all from w_i)
//   p_i = w_i - sum_k beta_k p_k,  s_i = A p_i
//   alpha = (p_i, r_i) / (p_i, s_i),  u += alpha p_i,  r -= alpha s_i
//   stop when ||r_{i+1}|| <= tol ||r_0|| (Table 1 criterion), or on breakdown
// Directions p_k and s_k = A p_k live in a ring of m_max+1 slots; slot(k) = k mod (m_max+1).
//
// Two implementations of the vector part:
//  - cluster: one thread-block cluster per instance (grids up to 128 x 128), each CTA holding a
//    band of 16 rows in registers (+ p in shared memory, halo rows from the neighbouring CTAs
//    through distributed shared memory); the step is one launch with fixed-order reductions;
//  - tiled: any N; seven launches per iteration (dots, beta, direction, stencil+dots,
//    alpha, update+norm, norm) with per-tile partial sums reduced in a fixed order.
// Both are deterministic: every sum has a fixed association order.
#include "internal.cuh"

#include <cooperative_groups.h>

#include <vector>
#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstring>

namespace fcgno {

constexpr int kTile = 2048;     // elements per CTA (tiled path)
constexpr int kThreads = 256;   // threads per CTA (tiled path)
constexpr int kEPT = kTile / kThreads;
constexpr int kParts = kMaxWindow + 2;
constexpr int kNarrowRunning = 80;  // running instances at or below which the narrow launch shape is used
constexpr int kTailRunning = 32;    // running instances at or below which a solve checks every kTailReplay
constexpr int kTailReplay = 2;      //   iterations (or check_every, if smaller)

struct IterArgs {
  int N;
  int B;
  size_t n;
  int tiles;
  int nslots;     // m_max + 1 ring slots
  double tol;
  int fixed;      // 1: ignore tol
};

// Iteration index and truncation window of one instance, derived on the device from that
// instance's own iteration count: captured CUDA graphs replay unchanged, and instances that
// started at different times (serving slots) can share a batch.
struct Window {
  int i;          // iteration index
  int m_i;        // window length min(i, max(1, i mod (m_max+1)))
  int slot_new;   // ring slot of p_i, s_i
  int slots[kMaxWindow];
};

struct State {
  const double* aE;
  const double* aN;
  const double* diag;
  const double* b;
  double* u;
  double* r;
  const double* w;
  double* P;
  double* S;
  double* ps;
  double* beta;
  double* alpha;
  double* r0;
  double* rr;
  double* rms;
  double* part;
  int* status;
  int* iters;
  int* ndone;
  int* iter;      // device iteration counter (advanced once per iteration)
};

__device__ __forceinline__ Window window_of(const IterArgs& a, const State& s, int b) {
  Window w;
  w.i = s.iters[b];
  w.m_i = min(w.i, max(1, w.i % a.nslots));
  w.slot_new = w.i % a.nslots;
#pragma unroll
  for (int j = 0; j < kMaxWindow; ++j) w.slots[j] = (j < w.m_i) ? (w.i - w.m_i + j) % a.nslots : 0;
  return w;
}



__device__ __forceinline__ double stencil_at(const State& s, size_t gi, int p, int q, int N, double c,
                                             double e, double w, double nn, double so) {
  // (A x)_P = diag x_P - aE_P x_E - aE_W x_W - aN_P x_N - aN_S x_S   (couplings pre-scaled)
  double acc = s.diag[gi] * c;
  if (p < N - 1) acc = fma(-s.aE[gi], e, acc);
  if (p > 0) acc = fma(-s.aE[gi - 1], w, acc);
  if (q < N - 1) acc = fma(-s.aN[gi], nn, acc);
  if (q > 0) acc = fma(-s.aN[gi - N], so, acc);
  return acc;
}

// Block-wide sums of the first `count` (<= NV) per-thread values, in a fixed order: the
// per-thread values go to shared memory; value j is summed by warp j mod (warps): each lane
// adds its strided share pairwise, then a 5-step shuffle tree combines the lanes. This costs
// about (blockDim/32 + 5) FP64 adds per lane of one warp per value instead of 5 per thread
// of the block. `sm` holds NV * blockDim doubles, `out` NV. Every thread gets the sums.
// Contains two __syncthreads().
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], int count, double* sm, double* out) {
  const int T = blockDim.x, nw = (T + 31) >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NV; ++j)
    if (j < count) sm[j * T + threadIdx.x] = v[j];
  __syncthreads();
  for (int j = warp; j < count; j += nw) {
    // lane sums elements lane, lane+32, ... (at most 32 of them) as a pairwise tree
    double loc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const int e = lane + 32 * t;
      loc[t] = (e < T) ? sm[j * T + e] : 0.0;
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
#pragma unroll
      for (int t = 0; t < w; ++t) loc[t] += loc[t + w];
    const double acc = warp_sum(loc[0]);
    if (lane == 0) out[j] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j)
    if (j < count) v[j] = out[j];
}

// ------------------------------------ initialisation -----------------------------------
// r_0 = b - A u_0, partial ||r_0||^2 per tile.
__global__ void __launch_bounds__(kThreads) init_kernel(IterArgs a, State s) {
  __shared__ double scratch[32];
  const int b = blockIdx.y;
  const size_t off = (size_t)b * a.n;
  double acc[1] = {0.0};
  for (int j = 0; j < kEPT; ++j) {
    const size_t e = (size_t)blockIdx.x * kTile + j * kThreads + threadIdx.x;
    if (e < a.n) {
      const int q = (int)(e / a.N), p = (int)(e - (size_t)q * a.N);
      const double* u = s.u + off;
      const double c = u[e];
      const double ue = (p < a.N - 1) ? u[e + 1] : 0.0;
      const double uw = (p > 0) ? u[e - 1] : 0.0;
      const double un = (q < a.N - 1) ? u[e + a.N] : 0.0;
      const double us = (q > 0) ? u[e - a.N] : 0.0;
      const double Au = stencil_at(s, off + e, p, q, a.N, c, ue, uw, un, us);
      const double rv = s.b[off + e] - Au;
      s.r[off + e] = rv;
      acc[0] = fma(rv, rv, acc[0]);
    }
  }
  const double tot = block_sum_lane<double, 1>(acc, 1, scratch);
  if (threadIdx.x == 0) s.part[((size_t)b * a.tiles + blockIdx.x) * kParts] = tot;
}

// Per-instance total of the first `count` tile partials (one block of kThreads per instance):
// thread i adds tiles i, i + kThreads, ... in order, then a fixed-order block reduction;
// returns the total of partial j in thread j (j < count).
template <int NV>
__device__ __forceinline__ double tile_totals(const IterArgs& a, const State& s, int b, int count, int first,
                                              double* scratch) {
  double v[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = 0.0;
  for (int t = threadIdx.x; t < a.tiles; t += blockDim.x) {
    const double* pp = s.part + ((size_t)b * a.tiles + t) * kParts + first;
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < count) v[j] += pp[j];
  }
  return block_sum_lane<double, NV>(v, count, scratch);
}

__global__ void __launch_bounds__(kThreads) init_finalize_kernel(IterArgs a, State s) {
  __shared__ double scratch[32];
  const int b = blockIdx.x;
  const double rr_t = tile_totals<1>(a, s, b, 1, 0, scratch);
  if (threadIdx.x != 0) return;
  const double rr = rr_t;
  s.rr[b] = rr;
  s.r0[b] = sqrt(rr);
  s.rms[b] = sqrt(rr / (double)a.n);
  s.iters[b] = 0;
  if (rr == 0.0) {
    s.status[b] = FCGNO_OK;
    atomicAdd(s.ndone, 1);
  } else {
    s.status[b] = kRunning;
  }
}

// ------------------------------------ tiled path ---------------------------------------
__global__ void __launch_bounds__(kThreads) dots_w_kernel(IterArgs a, State s) {
  __shared__ double scratch[32 * kMaxWindow];
  const int b = blockIdx.y;
  const Window w = window_of(a, s, b);
  if (s.status[b] != kRunning || w.m_i == 0) return;
  const size_t off = (size_t)b * a.n;
  // the tile's w values stay in registers; each window entry is a warp-uniform branch around
  // its own loads and FMAs (no FP64 work is issued for entries beyond m_i)
  const size_t e0 = (size_t)blockIdx.x * kTile + threadIdx.x;
  double wv[kEPT];
#pragma unroll
  for (int t = 0; t < kEPT; ++t) wv[t] = (e0 + t * kThreads < a.n) ? s.w[off + e0 + t * kThreads] : 0.0;
  double acc[kMaxWindow];
#pragma unroll
  for (int j = 0; j < kMaxWindow; ++j) {
    acc[j] = 0.0;
    if (j < w.m_i) {
      const double* Sj = s.S + (size_t)w.slots[j] * a.B * a.n + off + e0;
#pragma unroll
      for (int t = 0; t < kEPT; ++t)
        if (e0 + t * kThreads < a.n) acc[j] = fma(wv[t], Sj[t * kThreads], acc[j]);
    }
  }
  const double tot = block_sum_lane<double, kMaxWindow>(acc, w.m_i, scratch);
  if ((int)threadIdx.x < w.m_i) s.part[((size_t)b * a.tiles + blockIdx.x) * kParts + threadIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) beta_kernel(IterArgs a, State s) {
  __shared__ double scratch[32 * kMaxWindow];
  const int b = blockIdx.x;
  const int j = threadIdx.x;
  const Window w = window_of(a, s, b);
  if (s.status[b] != kRunning || w.m_i == 0) return;
  const double sum = tile_totals<kMaxWindow>(a, s, b, w.m_i, 0, scratch);
  if (j < w.m_i) s.beta[b * kMaxWindow + j] = sum / s.ps[(size_t)w.slots[j] * a.B + b];
}

__global__ void __launch_bounds__(kThreads) direction_kernel(IterArgs a, State s) {
  const int b = blockIdx.y;
  if (s.status[b] != kRunning) return;
  const Window w = window_of(a, s, b);
  const size_t off = (size_t)b * a.n;
  double beta[kMaxWindow];
#pragma unroll
  for (int j = 0; j < kMaxWindow; ++j) beta[j] = (j < w.m_i) ? s.beta[b * kMaxWindow + j] : 0.0;
  double* pn = s.P + (size_t)w.slot_new * a.B * a.n + off;
  const size_t e0 = (size_t)blockIdx.x * kTile + threadIdx.x;
  double pv[kEPT];
#pragma unroll
  for (int t = 0; t < kEPT; ++t) pv[t] = (e0 + t * kThreads < a.n) ? s.w[off + e0 + t * kThreads] : 0.0;
  // one warp-uniform branch per window entry (no FP64 work for entries beyond m_i)
#pragma unroll
  for (int j = 0; j < kMaxWindow; ++j) {
    if (j < w.m_i) {
      const double* Pj = s.P + (size_t)w.slots[j] * a.B * a.n + off + e0;
#pragma unroll
      for (int t = 0; t < kEPT; ++t)
        if (e0 + t * kThreads < a.n) pv[t] = fma(-beta[j], Pj[t * kThreads], pv[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < kEPT; ++t)
    if (e0 + t * kThreads < a.n) pn[e0 + t * kThreads] = pv[t];
}

__global__ void __launch_bounds__(kThreads) stencil_dots_kernel(IterArgs a, State s) {
  __shared__ double scratch[32 * 2];
  const int b = blockIdx.y;
  if (s.status[b] != kRunning) return;
  const Window w = window_of(a, s, b);
  const size_t off = (size_t)b * a.n;
  const double* pv = s.P + (size_t)w.slot_new * a.B * a.n + off;
  double* sv = s.S + (size_t)w.slot_new * a.B * a.n + off;
  double acc[2] = {0.0, 0.0};
  for (int t = 0; t < kEPT; ++t) {
    const size_t e = (size_t)blockIdx.x * kTile + t * kThreads + threadIdx.x;
    if (e < a.n) {
      const int q = (int)(e / a.N), p = (int)(e - (size_t)q * a.N);
      const double c = pv[e];
      const double ue = (p < a.N - 1) ? pv[e + 1] : 0.0;
      const double uw = (p > 0) ? pv[e - 1] : 0.0;
      const double un = (q < a.N - 1) ? pv[e + a.N] : 0.0;
      const double us = (q > 0) ? pv[e - a.N] : 0.0;
      const double Ap = stencil_at(s, off + e, p, q, a.N, c, ue, uw, un, us);
      sv[e] = Ap;
      acc[0] = fma(c, Ap, acc[0]);
      acc[1] = fma(c, s.r[off + e], acc[1]);
    }
  }
  const double tot = block_sum_lane<double, 2>(acc, 2, scratch);
  if (threadIdx.x < 2) s.part[((size_t)b * a.tiles + blockIdx.x) * kParts + threadIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) alpha_kernel(IterArgs a, State s) {
  __shared__ double scratch[32 * 2];
  __shared__ double pr_s;
  const int b = blockIdx.x;
  if (s.status[b] != kRunning) return;
  const Window w = window_of(a, s, b);
  const double tot = tile_totals<2>(a, s, b, 2, 0, scratch);
  if (threadIdx.x == 1) pr_s = tot;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double ps = tot, pr = pr_s;
  if (!(ps != 0.0 && isfinite(ps) && isfinite(pr))) {
    s.status[b] = FCGNO_EBREAKDOWN;
    atomicAdd(s.ndone, 1);
    return;
  }
  s.alpha[b] = pr / ps;
  s.ps[(size_t)w.slot_new * a.B + b] = ps;
}

__global__ void __launch_bounds__(kThreads) update_kernel(IterArgs a, State s) {
  __shared__ double scratch[32];
  const int b = blockIdx.y;
  if (s.status[b] != kRunning) return;
  const Window w = window_of(a, s, b);
  const size_t off = (size_t)b * a.n;
  const double alpha = s.alpha[b];
  const double* pv = s.P + (size_t)w.slot_new * a.B * a.n + off;
  const double* sv = s.S + (size_t)w.slot_new * a.B * a.n + off;
  double acc[1] = {0.0};
  for (int t = 0; t < kEPT; ++t) {
    const size_t e = (size_t)blockIdx.x * kTile + t * kThreads + threadIdx.x;
    if (e < a.n) {
      s.u[off + e] = fma(alpha, pv[e], s.u[off + e]);
      const double rv = fma(-alpha, sv[e], s.r[off + e]);
      s.r[off + e] = rv;
      acc[0] = fma(rv, rv, acc[0]);
    }
  }
  const double tot = block_sum_lane<double, 1>(acc, 1, scratch);
  if (threadIdx.x == 0) s.part[((size_t)b * a.tiles + blockIdx.x) * kParts + 2] = tot;
}

__global__ void __launch_bounds__(kThreads) norm_kernel(IterArgs a, State s) {
  __shared__ double scratch[32];
  const int b = blockIdx.x;
  if (s.status[b] != kRunning) return;
  const Window w = window_of(a, s, b);
  const double rr_t = tile_totals<1>(a, s, b, 1, 2, scratch);
  if (threadIdx.x != 0) return;
  const double rr = rr_t;
  s.rr[b] = rr;
  s.rms[b] = sqrt(rr / (double)a.n);
  s.iters[b] = w.i + 1;
  const double rn = sqrt(rr);
  if (rr == 0.0 || (!a.fixed && rn <= a.tol * s.r0[b])) {
    s.status[b] = FCGNO_OK;
    atomicAdd(s.ndone, 1);
  }
}

// ------------------------------------ cluster path -------------------------------------
// One thread-block cluster of CL CTAs per instance (N <= kClusterMaxN). CTA c owns the grid rows
// [c*band, min(N, (c+1)*band)); thread t owns the band's elements t + j*blockDim (j < EPT).
// The instance's FP64 work is spread over CL SMs: GB300 runs about 2 FP64 multiply-adds per
// clock per SM, so one SM per instance would bound a 64 x 64 step to ~20 us on its own.
// Each sum is a fixed-order block reduction per CTA followed by the CL partials summed in rank
// order, read through distributed shared memory; every CTA forms the same totals, so the
// per-instance decisions (breakdown, convergence) are taken identically across the cluster.
// The stencil's halo rows are copied from the neighbouring CTAs' shared memory after a cluster
// barrier. A final cluster barrier keeps every CTA resident until the others have read its
// partial sums.
constexpr int kClusterThreads = 256;
constexpr int kClusterBand = 16;   // grid rows per CTA
constexpr int kClusterMaxN = 128;  // kClusterBand * N <= 8 * kClusterThreads and CL <= 8
constexpr int kWideMaxN = 80;      // one CTA per instance: n / 8 <= 1024 threads

template <int EPT, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT > 256 ? 1 : (EPT >= 8 ? 2 : 4)) cluster_step_kernel(IterArgs a, State s,
                                                                                                 int band) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double smc[];  // (band + 2) * N doubles of p (halo row, band rows, halo row),
                                   // then kMaxWindow * blockDim doubles (block reductions)
  __shared__ double part[3][kMaxWindow];  // this CTA's partial sums: window dots; (p,s),(p,r); ||r||^2
  __shared__ double red_out[kMaxWindow];
  __shared__ double beta_s[kMaxWindow];
  pdl_wait();
  pdl_trigger();
  const int CL = (int)cl.num_blocks(), c = (int)cl.block_rank();
  // a cluster of one CTA synchronises and reads its partial sums as a plain block
  auto csync = [&]() {
    if (CL > 1)
      cl.sync();
    else
      __syncthreads();
  };
  auto at = [&](double* ptr, int rank) -> const double* { return rank == c ? ptr : cl.map_shared_rank(ptr, rank); };
  const int b = blockIdx.x / CL;
  if (s.status[b] != kRunning) return;  // the same for every CTA of the cluster
  const Window wd = window_of(a, s, b);
  const int N = a.N, T = blockDim.x;
  const int q0 = c * band, q1 = min(N, q0 + band);
  const int nb = (q1 - q0) * N;  // elements of this CTA
  const size_t off = (size_t)b * a.n + (size_t)q0 * N;
  double* ph = smc;                     // ph[N + e] = p of band element e; rows 0 and band+1 are halos
  double* red = smc + (size_t)(band + 2) * N;
  double wv[EPT], sv[EPT];  // r is re-read in the update (it is still in L1): fewer live registers
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = threadIdx.x + j * T;
    wv[j] = (e < nb) ? s.w[off + e] : 0.0;
  }
  // beta_k = (w, s_k) / (p_k, s_k)
  double acc[kMaxWindow];
#pragma unroll
  for (int k = 0; k < kMaxWindow; ++k) {
    acc[k] = 0.0;
    if (k < wd.m_i) {
      const double* Sk = s.S + (size_t)wd.slots[k] * a.B * a.n + off;
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const int e = threadIdx.x + j * T;
        if (e < nb) acc[k] = fma(wv[j], Sk[e], acc[k]);
      }
    }
  }
  if (wd.m_i > 0) {
    block_sums<kMaxWindow>(acc, wd.m_i, red, red_out);
    if ((int)threadIdx.x < wd.m_i) {
      double v = acc[0];
#pragma unroll
      for (int k = 1; k < kMaxWindow; ++k)
        if ((int)threadIdx.x == k) v = acc[k];
      part[0][threadIdx.x] = v;
    }
  }
  csync();  // (1) window partials
  if ((int)threadIdx.x < wd.m_i) {
    double tot = 0.0;
    for (int r = 0; r < CL; ++r) tot += at(&part[0][0], r)[threadIdx.x];
    beta_s[threadIdx.x] = tot / s.ps[(size_t)wd.slots[threadIdx.x] * a.B + b];
  }
  __syncthreads();
  // p = w - sum beta_k p_k (kept in wv)
#pragma unroll
  for (int k = 0; k < kMaxWindow; ++k) {
    if (k < wd.m_i) {
      const double beta = beta_s[k];
      const double* Pk = s.P + (size_t)wd.slots[k] * a.B * a.n + off;
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const int e = threadIdx.x + j * T;
        if (e < nb) wv[j] = fma(-beta, Pk[e], wv[j]);
      }
    }
  }
  double* Pn = s.P + (size_t)wd.slot_new * a.B * a.n + off;
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = threadIdx.x + j * T;
    if (e < nb) {
      ph[N + e] = wv[j];
      Pn[e] = wv[j];
    }
  }
  csync();  // (2) every band of p in shared memory
  // halo rows: the last row of the CTA above, the first row of the CTA below (zero at the walls)
  for (int i = threadIdx.x; i < 2 * N; i += T) {
    const int p = i % N;
    if (i < N) {
      ph[p] = (c > 0) ? at(ph, c - 1)[N + (band - 1) * N + p] : 0.0;
    } else {
      ph[(size_t)(q1 - q0 + 1) * N + p] = (q1 < N) ? at(ph, c + 1)[N + p] : 0.0;
    }
  }
  __syncthreads();
  // s = A p, (p, s), (p, r)
  double d2[2] = {0.0, 0.0};
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = threadIdx.x + j * T;
    sv[j] = 0.0;
    if (e < nb) {
      const int ql = e / N, p = e - ql * N;
      const double* row = ph + (size_t)(ql + 1) * N;
      const double ue = (p < N - 1) ? row[p + 1] : 0.0;
      const double uw = (p > 0) ? row[p - 1] : 0.0;
      // halo rows carry the neighbour's p, or zero at the Dirichlet walls
      sv[j] = stencil_at(s, off + e, p, q0 + ql, N, wv[j], ue, uw, row[p + N], row[p - N]);
      d2[0] = fma(wv[j], sv[j], d2[0]);
      d2[1] = fma(wv[j], s.r[off + e], d2[1]);
    }
  }
  block_sums<2>(d2, 2, red, red_out);
  if (threadIdx.x == 0) {
    part[1][0] = d2[0];
    part[1][1] = d2[1];
  }
  csync();  // (3) (p, s), (p, r) partials
  double ps = 0.0, pr = 0.0;
  for (int r = 0; r < CL; ++r) {
    const double* pp = at(&part[1][0], r);
    ps += pp[0];
    pr += pp[1];
  }
  const bool broke = !(ps != 0.0 && isfinite(ps) && isfinite(pr));
  double rr = 0.0;
  if (!broke) {
    const double alpha = pr / ps;
    double* Sn = s.S + (size_t)wd.slot_new * a.B * a.n + off;
    double r2[1] = {0.0};
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      const int e = threadIdx.x + j * T;
      if (e < nb) {
        Sn[e] = sv[j];
        s.u[off + e] = fma(alpha, wv[j], s.u[off + e]);
        const double r1 = fma(-alpha, sv[j], s.r[off + e]);
        s.r[off + e] = r1;
        r2[0] = fma(r1, r1, r2[0]);
      }
    }
    block_sums<1>(r2, 1, red, red_out);
    if (threadIdx.x == 0) part[2][0] = r2[0];
  }
  csync();  // (4) ||r||^2 partials (unused after a breakdown)
  if (!broke) {
    for (int r = 0; r < CL; ++r) rr += at(&part[2][0], r)[0];
  }
  if (c == 0 && threadIdx.x == 0) {
    if (broke) {
      s.status[b] = FCGNO_EBREAKDOWN;
      atomicAdd(s.ndone, 1);
    } else {
      s.ps[(size_t)wd.slot_new * a.B + b] = ps;
      s.alpha[b] = pr / ps;
      s.rr[b] = rr;
      s.rms[b] = sqrt(rr / (double)a.n);
      s.iters[b] = wd.i + 1;
      if (rr == 0.0 || (!a.fixed && sqrt(rr) <= a.tol * s.r0[b])) {
        s.status[b] = FCGNO_OK;
        atomicAdd(s.ndone, 1);
      }
    }
  }
  csync();  // (5) no CTA leaves while another still reads its shared memory
}

// FP64 multiply-add rate (a measurement aid, not a step of the method). Every thread runs
// kRateChains independent chains x <- fma(x, a, c), started at x = 1 + j/16, for `steps`
// steps, and writes the sum of its chains' final values. The chains keep enough independent
// multiply-adds in flight to fill the FP64 pipe; nothing else is in the loop.
constexpr int kRateChains = 8;
constexpr int kRateThreads = 256;
__global__ void __launch_bounds__(kRateThreads) fp64_fma_rate_kernel(int steps, double a, double c,
                                                                    double* __restrict__ out) {
  double x[kRateChains];
#pragma unroll
  for (int j = 0; j < kRateChains; ++j) x[j] = 1.0 + 0.0625 * j;
  for (int t = 0; t < steps; ++t) {
#pragma unroll
    for (int j = 0; j < kRateChains; ++j) x[j] = fma(x[j], a, c);
  }
  double sum = 0.0;
#pragma unroll
  for (int j = 0; j < kRateChains; ++j) sum += x[j];
  out[(size_t)blockIdx.x * kRateThreads + threadIdx.x] = sum;
}

// Jacobi(k) preconditioner, Eq. (15): x_0 = 0, x_{j+1} = x_j + D^-1 (r - A x_j); the first
// sweep reduces to D^-1 r. x_in == nullptr marks the first sweep.
__global__ void inv_diag_kernel(size_t total, const double* __restrict__ diag, double* __restrict__ inv) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < total) inv[i] = 1.0 / diag[i];
}

__global__ void jacobi_sweep_kernel(int N, size_t n, const int* __restrict__ status, const double* __restrict__ aE,
                                    const double* __restrict__ aN, const double* __restrict__ diag,
                                    const double* __restrict__ inv, const double* __restrict__ r,
                                    const double* __restrict__ xin, double* __restrict__ xout) {
  const int b = blockIdx.y;
  if (status[b] != kRunning) return;
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const size_t gi = (size_t)b * n + e;
  if (!xin) {
    xout[gi] = r[gi] * inv[gi];
    return;
  }
  const int q = (int)(e / N), p = (int)(e - (size_t)q * N);
  double Ax = diag[gi] * xin[gi];
  if (p < N - 1) Ax = fma(-aE[gi], xin[gi + 1], Ax);
  if (p > 0) Ax = fma(-aE[gi - 1], xin[gi - 1], Ax);
  if (q < N - 1) Ax = fma(-aN[gi], xin[gi + N], Ax);
  if (q > 0) Ax = fma(-aN[gi - N], xin[gi - N], Ax);
  xout[gi] = fma(r[gi] - Ax, inv[gi], xin[gi]);
}

// Krylov sampling helper: r_out[i] = r, e_out[i] = u_star - u for every instance.
__global__ void harvest_copy_kernel(size_t total, const double* __restrict__ r, const double* __restrict__ u,
                                    const double* __restrict__ ustar, double* __restrict__ r_out,
                                    double* __restrict__ e_out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  r_out[i] = r[i];
  e_out[i] = ustar[i] - u[i];
}

// ------------------------------------ host side ----------------------------------------
static void drop_graph(IterGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  trace_release(g.traced);
  g = IterGraph();
}

static void drop_graph(SolverWorkspace& w) {
  for (IterGraph& g : w.graph) drop_graph(g);
}

static void free_ws(SolverWorkspace& w) {
  drop_graph(w);
  double** dp[] = {&w.r, &w.w, &w.wt, &w.inv_diag, &w.P, &w.S, &w.ps, &w.beta, &w.alpha, &w.r0, &w.rr, &w.rms, &w.part};
  for (auto p : dp) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  int** ip[] = {&w.status, &w.iters, &w.ndone, &w.iter};
  for (auto p : ip) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  w.cap_B = w.cap_n = w.cap_slots = w.cap_tiles = 0;
}

void solver_ws_free(fcgno_op* op) {
  free_ws(op->ws);
  if (op->ws.cs) cudaStreamDestroy(op->ws.cs);
  if (op->ws.ev_in) cudaEventDestroy(op->ws.ev_in);
  if (op->ws.ev_out) cudaEventDestroy(op->ws.ev_out);
  op->ws.cs = nullptr;
  op->ws.ev_in = op->ws.ev_out = nullptr;
}

// Byte sizes of the solver workspace's device buffers, in the order ensure_ws allocates them
// (r, w, wt, inv_diag, P, S, ps, beta, alpha, r0, rr, rms, part, status, iters, ndone, iter).
// fcgno_workspace_bytes sums the same list, so admission counts exactly what is allocated.
constexpr int kWsBuffers = 17;
static void solver_ws_sizes(size_t n, int B, int slots, size_t (&sz)[kWsBuffers]) {
  const size_t vec = n * B * sizeof(double);
  const size_t tiles = ceil_div(n, kTile);
  const size_t list[kWsBuffers] = {vec, vec, vec, vec, vec * slots, vec * slots,
                                   sizeof(double) * slots * B, sizeof(double) * kMaxWindow * B,
                                   sizeof(double) * B, sizeof(double) * B, sizeof(double) * B, sizeof(double) * B,
                                   sizeof(double) * B * tiles * kParts, sizeof(int) * B, sizeof(int) * B,
                                   sizeof(int), sizeof(int)};
  for (int i = 0; i < kWsBuffers; ++i) sz[i] = list[i];
}

size_t solver_ws_bytes(size_t n, int B, int slots) {
  size_t sz[kWsBuffers];
  solver_ws_sizes(n, B, slots, sz);
  size_t t = 0;
  for (size_t v : sz) t += v;
  return t;
}

static fcgno_status ensure_ws(fcgno_op* op, int slots) {
  SolverWorkspace& w = op->ws;
  if (!w.cs) {
    FCGNO_CUDA_TRY(cudaStreamCreateWithFlags(&w.cs, cudaStreamNonBlocking));
    FCGNO_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_in, cudaEventDisableTiming));
    FCGNO_CUDA_TRY(cudaEventCreateWithFlags(&w.ev_out, cudaEventDisableTiming));
  }
  const int tiles = (int)ceil_div(op->n, kTile);
  if (w.cap_B == op->B && w.cap_n == (int)op->n && w.cap_slots >= slots && w.cap_tiles >= tiles) return FCGNO_OK;
  free_ws(w);
  size_t sz[kWsBuffers];
  solver_ws_sizes(op->n, op->B, slots, sz);
  void** bufs[kWsBuffers] = {(void**)&w.r,     (void**)&w.w,     (void**)&w.wt,     (void**)&w.inv_diag,
                             (void**)&w.P,     (void**)&w.S,     (void**)&w.ps,     (void**)&w.beta,
                             (void**)&w.alpha, (void**)&w.r0,    (void**)&w.rr,     (void**)&w.rms,
                             (void**)&w.part,  (void**)&w.status, (void**)&w.iters, (void**)&w.ndone,
                             (void**)&w.iter};
  bool ok = true;
  for (int i = 0; i < kWsBuffers && ok; ++i)
    if (cudaMalloc(bufs[i], sz[i]) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    free_ws(w);
    set_last_error("solver workspace: out of device memory");
    return FCGNO_ENOMEM;
  }
  w.cap_B = op->B;
  w.cap_n = (int)op->n;
  w.cap_slots = slots;
  w.cap_tiles = tiles;
  return FCGNO_OK;
}

static State make_state(fcgno_op* op, const double* b, double* x, const double* wptr) {
  SolverWorkspace& w = op->ws;
  State s;
  s.aE = op->aE;
  s.aN = op->aN;
  s.diag = op->diag;
  s.b = b;
  s.u = x;
  s.r = w.r;
  s.w = wptr;
  s.P = w.P;
  s.S = w.S;
  s.ps = w.ps;
  s.beta = w.beta;
  s.alpha = w.alpha;
  s.r0 = w.r0;
  s.rr = w.rr;
  s.rms = w.rms;
  s.part = w.part;
  s.status = w.status;
  s.iters = w.iters;
  s.ndone = w.ndone;
  s.iter = w.iter;
  return s;
}

struct HarvestHook {
  const double* ustar = nullptr;
  double* r_out = nullptr;
  double* e_out = nullptr;
};

struct LoopShape {
  bool cluster;      // N <= kClusterMaxN: the step is one launch of cluster_step_kernel
  int CL;            // CTAs per instance (cluster size)
  int band;          // grid rows per CTA
  int EPT;           // elements per thread
  int threads;       // threads per CTA
  bool big;          // threads > 256 (the 1024-thread instantiation)
  size_t smem;       // dynamic shared memory per CTA
};

// Launch shape of the FCG step. Wide (many instances running): for N <= 80 one CTA holds a whole
// instance (8 elements per thread, up to 1024 threads), which keeps the FP64 pipe of every SM
// busy with few synchronisations; larger N and the narrow shape (few instances running) split
// each instance over a cluster of 16-row bands on 256-thread CTAs, so that one instance's step
// runs on several SMs.
static LoopShape loop_shape(const fcgno_op* op, bool narrow = false) {
  LoopShape L{};
  L.cluster = op->N <= kClusterMaxN;
  if (!L.cluster) return L;
  const int N = op->N;
  if (!narrow && N <= kWideMaxN) {
    L.CL = 1;
    L.band = N;
    L.EPT = 8;
    L.threads = (int)((ceil_div(op->n, 8) + 31) / 32 * 32);
  } else {
    L.band = std::min(kClusterBand, N);
    L.CL = (N + L.band - 1) / L.band;
    const int need = (L.band * N + kClusterThreads - 1) / kClusterThreads;
    L.EPT = need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : 8;
    L.threads = kClusterThreads;
  }
  L.big = L.threads > kClusterThreads;
  L.smem = ((size_t)(L.band + 2) * N + (size_t)kMaxWindow * L.threads) * sizeof(double);
  return L;
}

template <int EPT, int MAXT>
static fcgno_status prepare_cluster_kernel(size_t smem) {
  const void* fn = (const void*)cluster_step_kernel<EPT, MAXT>;
  if (smem > 48 * 1024)
    FCGNO_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FCGNO_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
  return FCGNO_OK;
}

// Raise the step kernel's shared-memory limit before its first launch (not a stream
// operation, so it stays outside graph capture).
static fcgno_status prepare_fused(const LoopShape& L) {
  if (!L.cluster) return FCGNO_OK;
  if (L.big) return prepare_cluster_kernel<8, 1024>(L.smem);
  switch (L.EPT) {
    case 1: return prepare_cluster_kernel<1, kClusterThreads>(L.smem);
    case 2: return prepare_cluster_kernel<2, kClusterThreads>(L.smem);
    case 4: return prepare_cluster_kernel<4, kClusterThreads>(L.smem);
    default: return prepare_cluster_kernel<8, kClusterThreads>(L.smem);
  }
}

template <int EPT, int MAXT>
static cudaError_t launch_cluster_step(const IterArgs& a, const State& s, const LoopShape& L, cudaStream_t cs) {
  return launch_chained_cluster(cluster_step_kernel<EPT, MAXT>, dim3(L.CL * a.B), dim3(L.threads), L.smem, cs,
                                L.CL, a, s, L.band);
}

// The vector part of one iteration (steps a3-a7) plus the iteration-counter advance.
static fcgno_status launch_vector_step(const IterArgs& a, const State& s, const LoopShape& L, cudaStream_t cs) {
  if (L.cluster) {
    {
      TraceScope ts("fcg_fused", cs);
      cudaError_t e;
      if (L.big) {
        e = launch_cluster_step<8, 1024>(a, s, L, cs);
      } else {
        switch (L.EPT) {
          case 1: e = launch_cluster_step<1, kClusterThreads>(a, s, L, cs); break;
          case 2: e = launch_cluster_step<2, kClusterThreads>(a, s, L, cs); break;
          case 4: e = launch_cluster_step<4, kClusterThreads>(a, s, L, cs); break;
          default: e = launch_cluster_step<8, kClusterThreads>(a, s, L, cs); break;
        }
      }
      if (e != cudaSuccess) {
        set_last_error(std::string("cluster step launch: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return FCGNO_ECUDA;
      }
    }
    FCGNO_LAUNCHED();
  } else {
    TraceScope ts("fcg_tiled", cs);
    const dim3 grid(a.tiles, a.B);
    dots_w_kernel<<<grid, kThreads, 0, cs>>>(a, s);
    FCGNO_LAUNCHED();
    beta_kernel<<<a.B, kThreads, 0, cs>>>(a, s);
    FCGNO_LAUNCHED();
    direction_kernel<<<grid, kThreads, 0, cs>>>(a, s);
    FCGNO_LAUNCHED();
    stencil_dots_kernel<<<grid, kThreads, 0, cs>>>(a, s);
    FCGNO_LAUNCHED();
    alpha_kernel<<<a.B, kThreads, 0, cs>>>(a, s);
    FCGNO_LAUNCHED();
    update_kernel<<<grid, kThreads, 0, cs>>>(a, s);
    FCGNO_LAUNCHED();
    norm_kernel<<<a.B, kThreads, 0, cs>>>(a, s);
    FCGNO_LAUNCHED();
  }
  return FCGNO_OK;
}

static fcgno_status launch_jacobi(fcgno_op* op, int steps, cudaStream_t cs) {
  SolverWorkspace& w = op->ws;
  // sweeps alternate between w and wt so that the last one lands in w
  double* bufs[2] = {w.w, w.wt};
  int cur = (steps % 2 == 1) ? 0 : 1;
  const double* xin = nullptr;
  for (int j = 0; j < steps; ++j) {
    double* xout = bufs[cur];
    jacobi_sweep_kernel<<<dim3(ceil_div(op->n, 256), op->B), 256, 0, cs>>>(op->N, op->n, w.status, op->aE, op->aN,
                                                                          op->diag, w.inv_diag, w.r, xin, xout);
    FCGNO_LAUNCHED();
    xin = xout;
    cur ^= 1;
  }
  return FCGNO_OK;
}

struct ServeDev;
static fcgno_status launch_serve(const ServeDev& v, const IterArgs& a, const State& s, cudaStream_t cs);

static fcgno_status launch_iteration(fcgno_op* op, fcgno_model* model, fcgno_prec prec, const IterArgs& a,
                                     const State& s, const LoopShape& L, cudaStream_t cs, int jacobi = 0,
                                     bool narrow = false, const ServeDev* serve = nullptr) {
  if (serve) FCGNO_TRY(launch_serve(*serve, a, s, cs));
  if (jacobi > 0) {
    FCGNO_TRY(launch_jacobi(op, jacobi, cs));
  } else if (model) {
    SolverWorkspace& w = op->ws;
    if (prec == FCGNO_BF16 || prec == FCGNO_FP16) {
      FCGNO_TRY(no_apply_tc(model, op, w.r, w.rms, w.status, w.w, prec == FCGNO_FP16, cs, narrow));
    } else {
      FCGNO_TRY(no_apply_simt(model, op, w.r, w.rms, w.status, w.w, prec == FCGNO_FP64, cs));
    }
  }
  return launch_vector_step(a, s, L, cs);
}

// Captures G iterations into a CUDA graph (reused while the baked-in parameters match).
static fcgno_status ensure_graph(fcgno_op* op, fcgno_model* model, fcgno_prec prec, const IterArgs& a,
                                 const State& s, const LoopShape& L, const double* b, const double* x, int G,
                                 int jacobi, bool narrow = false, const ServeDev* serve = nullptr, int slot = -1) {
  SolverWorkspace& w = op->ws;
  IterGraph& g = w.graph[slot >= 0 ? slot : (narrow ? 1 : 0)];
  const uint64_t gen = model ? model->gen : 0;
  if (g.exec && g.trace_gen == trace_generation() && g.model == model && g.model_gen == gen &&
      g.prec == (int)prec && g.nslots == a.nslots && g.jacobi == jacobi &&
      g.fixed == a.fixed && g.G == G && g.tol == a.tol && g.b == b && g.x == x && g.serve == serve)
    return FCGNO_OK;
  drop_graph(g);
  const uint64_t l0 = g_launches.load();
  FCGNO_CUDA_TRY(cudaStreamBeginCapture(w.cs, cudaStreamCaptureModeThreadLocal));
  trace_capture_begin(&g.traced);
  fcgno_status rc = FCGNO_OK;
  for (int it = 0; it < G && rc == FCGNO_OK; ++it)
    rc = launch_iteration(op, model, prec, a, s, L, w.cs, jacobi, narrow, serve);
  trace_capture_end();
  // captured launches did not run: they are counted when the graph replays
  g.kernels = g_launches.load() - l0;
  g_launches.fetch_sub(g.kernels);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(w.cs, &graph);
  if (rc != FCGNO_OK || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    trace_release(g.traced);
    if (rc == FCGNO_OK) {
      set_last_error(std::string("graph capture: ") + cudaGetErrorString(ec));
      rc = FCGNO_ECUDA;
    }
    return rc;
  }
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    g.exec = nullptr;
    trace_release(g.traced);
    set_last_error(std::string("graph instantiate: ") + cudaGetErrorString(ei));
    return FCGNO_ECUDA;
  }
  g.trace_gen = trace_generation();
  g.jacobi = jacobi;
  g.model = model;
  g.model_gen = gen;
  g.prec = (int)prec;
  g.nslots = a.nslots;
  g.fixed = a.fixed;
  g.G = G;
  g.tol = a.tol;
  g.b = b;
  g.x = x;
  g.serve = serve;
  return FCGNO_OK;
}

static bool graphs_enabled() {
  const char* e = getenv("FCGNO_GRAPHS");
  return !(e && e[0] == '0');
}

static fcgno_status solve_impl(fcgno_op* op, fcgno_model* model, const double* b, double* x,
                               const fcgno_solve_opts& o, fcgno_prec prec, fcgno_solve_info* info,
                               cudaStream_t st, const HarvestHook* hook, int jacobi = 0) {
  const int slots = o.m_max + 1;
  FCGNO_TRY(ensure_ws(op, slots));
  SolverWorkspace& w = op->ws;
  const cudaStream_t cs = w.cs;
  const bool identity = (model == nullptr && jacobi == 0);
  // with the identity preconditioner w_i = r_i: read r in place of w
  State s = make_state(op, b, x, identity ? w.r : w.w);
  IterArgs a{};
  a.N = op->N;
  a.B = op->B;
  a.n = op->n;
  a.tiles = (int)ceil_div(op->n, kTile);
  a.nslots = slots;
  a.tol = o.tol;
  a.fixed = o.fixed_iters ? 1 : 0;
  const LoopShape L = loop_shape(op), Ln = loop_shape(op, true);
  FCGNO_TRY(prepare_fused(L));
  FCGNO_TRY(prepare_fused(Ln));
  // the caller's stream orders our internal stream at entry and exit
  FCGNO_CUDA_TRY(cudaEventRecord(w.ev_in, st));
  FCGNO_CUDA_TRY(cudaStreamWaitEvent(cs, w.ev_in, 0));
  FCGNO_CUDA_TRY(cudaMemsetAsync(w.ndone, 0, sizeof(int), cs));
  FCGNO_CUDA_TRY(cudaMemsetAsync(w.iter, 0, sizeof(int), cs));
  init_kernel<<<dim3(a.tiles, op->B), kThreads, 0, cs>>>(a, s);
  FCGNO_LAUNCHED();
  init_finalize_kernel<<<op->B, kThreads, 0, cs>>>(a, s);
  FCGNO_LAUNCHED();
  if (jacobi > 0) {
    inv_diag_kernel<<<ceil_div(op->n * op->B, 256), 256, 0, cs>>>(op->n * op->B, op->diag, w.inv_diag);
    FCGNO_LAUNCHED();
  }

  int* h_ndone = nullptr;
  FCGNO_CUDA_TRY(cudaMallocHost(&h_ndone, sizeof(int)));
  struct PinnedGuard {
    int* p;
    ~PinnedGuard() { cudaFreeHost(p); }
  } guard{h_ndone};
  const int G = std::max(1, o.check_every);
  const bool use_graph = !hook && graphs_enabled() && G > 1;
  // once few instances are still running, the replayed iterations switch to the narrow launch
  // shapes (more blocks per instance, for the FCG step and the 16-bit preconditioner's
  // synthesis): the launches are then bound by one instance's serial chain, not by the batch's work
  const bool tc = model && (prec == FCGNO_BF16 || prec == FCGNO_FP16);
  const bool can_narrow = (tc && tc_has_narrow(op->N, model->desc)) || Ln.CL != L.CL;
  int running = op->B;
  int i = 0;
  int since_check = 0;
  int last_graph = 0;
  // the tail of a batch (few instances left, converging over a few iterations) replays
  // shorter graphs, so that the solve ends closer to the last instance's convergence
  const int Gt = std::min(G, kTailReplay);
  int curG = G;
  while (i < o.max_iter) {
    bool replayed = false;
    const bool tail = Gt < G && running <= kTailRunning;
    const int Gx = tail ? Gt : G;
    if (use_graph && i > 0 && o.max_iter - i >= Gx) {
      // the first iteration ran eagerly, so every lazily allocated buffer exists before capture
      const int mode = launch_shape_mode();
      const bool narrow = mode == 2 || (mode == 0 && can_narrow && running <= kNarrowRunning);
      last_graph = (narrow ? 1 : 0) + (tail ? 2 : 0);
      FCGNO_TRY(ensure_graph(op, model, prec, a, s, narrow ? Ln : L, b, x, Gx, jacobi, narrow, nullptr, last_graph));
      FCGNO_CUDA_TRY(cudaGraphLaunch(w.graph[last_graph].exec, cs));
      g_launches.fetch_add(w.graph[last_graph].kernels, std::memory_order_relaxed);
      i += Gx;
      since_check = Gx;
      curG = Gx;
      replayed = true;
    } else {
      const bool narrow = launch_shape_mode() == 2;
      FCGNO_TRY(launch_iteration(op, model, prec, a, s, narrow ? Ln : L, cs, jacobi, narrow));
      if (hook) {
        const size_t total = op->n * op->B;
        const size_t o2 = (size_t)i * total;
        harvest_copy_kernel<<<ceil_div(total, 256), 256, 0, cs>>>(total, w.r, x, hook->ustar, hook->r_out + o2,
                                                                  hook->e_out + o2);
        FCGNO_LAUNCHED();
      }
      ++i;
      ++since_check;
      curG = Gx;
    }
    if (since_check >= curG || i >= o.max_iter || (use_graph && i == 1)) {
      since_check = 0;
      FCGNO_CUDA_TRY(cudaMemcpyAsync(h_ndone, w.ndone, sizeof(int), cudaMemcpyDeviceToHost, cs));
      FCGNO_CUDA_TRY(cudaStreamSynchronize(cs));
      if (replayed) trace_accumulate(w.graph[last_graph].traced);
      running = op->B - *h_ndone;
      if (*h_ndone >= op->B && !hook) break;
    }
  }
  if (info) {
    std::vector<int> hs(op->B), hi(op->B);
    std::vector<double> hrr(op->B), hr0(op->B);
    FCGNO_CUDA_TRY(cudaMemcpyAsync(hs.data(), w.status, sizeof(int) * op->B, cudaMemcpyDeviceToHost, cs));
    FCGNO_CUDA_TRY(cudaMemcpyAsync(hi.data(), w.iters, sizeof(int) * op->B, cudaMemcpyDeviceToHost, cs));
    FCGNO_CUDA_TRY(cudaMemcpyAsync(hrr.data(), w.rr, sizeof(double) * op->B, cudaMemcpyDeviceToHost, cs));
    FCGNO_CUDA_TRY(cudaMemcpyAsync(hr0.data(), w.r0, sizeof(double) * op->B, cudaMemcpyDeviceToHost, cs));
    FCGNO_CUDA_TRY(cudaStreamSynchronize(cs));
    for (int bi = 0; bi < op->B; ++bi) {
      info[bi].iters = hi[bi];
      int stt = hs[bi];
      if (stt == kRunning) stt = o.fixed_iters ? FCGNO_OK : FCGNO_ENOCONV;
      info[bi].status = stt;
      info[bi].r0norm = hr0[bi];
      info[bi].relres = hr0[bi] > 0 ? std::sqrt(hrr[bi]) / hr0[bi] : 0.0;
    }
  } else {
    FCGNO_CUDA_TRY(cudaStreamSynchronize(cs));
  }
  FCGNO_CUDA_TRY(cudaEventRecord(w.ev_out, cs));
  FCGNO_CUDA_TRY(cudaStreamWaitEvent(st, w.ev_out, 0));
  return tc_take_timeout(op, cs);
}

static fcgno_status check_opts(const fcgno_solve_opts* o) {
  if (!o || !(o->tol >= 0.0) || o->m_max < 1 || o->m_max > kMaxWindow || o->max_iter < 0) {
    set_last_error("fcgno_solve: need tol >= 0, 1 <= m_max <= 8, max_iter >= 0");
    return FCGNO_EINVAL;
  }
  return FCGNO_OK;
}

}  // namespace fcgno

using namespace fcgno;

// Checks shared by the solve entry points, made before any allocation or launch: the
// options, the precision, and the preconditioner's shape on an N x N grid.
static fcgno_status check_solve_args(const char* who, int N, const fcgno_model* Bpc, const fcgno_solve_opts* opts,
                                     fcgno_prec prec) {
  FCGNO_TRY(check_opts(opts));
  if (prec < FCGNO_FP64 || prec > FCGNO_FP32) {
    set_last_error(std::string(who) + ": unknown precision");
    return FCGNO_EINVAL;
  }
  if (Bpc && N < 2 * Bpc->desc.modes) {
    set_last_error(std::string(who) + ": grid smaller than 2*modes");
    return FCGNO_EINVAL;
  }
  if (Bpc && (prec == FCGNO_BF16 || prec == FCGNO_FP16) && !tc_shape_supported(N, Bpc->desc)) {
    set_last_error(std::string(who) + ": " + tc_shape_rule());
    return FCGNO_EINVAL;
  }
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_solve(fcgno_op_t A, fcgno_model_t Bpc, const double* b, double* x,
                                    const fcgno_solve_opts* opts, fcgno_prec prec, fcgno_solve_info* info,
                                    void* stream) {
  if (!A || !b || !x) {
    set_last_error("fcgno_solve: null operator, b or x");
    return FCGNO_EINVAL;
  }
  FCGNO_TRY(check_solve_args("fcgno_solve", A->N, Bpc, opts, prec));
  return solve_impl(A, Bpc, b, x, *opts, prec, info, (cudaStream_t)stream, nullptr);
}

extern "C" fcgno_status fcgno_solve_jacobi(fcgno_op_t A, int steps, const double* b, double* x,
                                           const fcgno_solve_opts* opts, fcgno_solve_info* info, void* stream) {
  if (!A || !b || !x || steps < 1 || steps > 64) {
    set_last_error("fcgno_solve_jacobi: null operator, b or x, or steps outside 1..64");
    return FCGNO_EINVAL;
  }
  FCGNO_TRY(check_opts(opts));
  return solve_impl(A, nullptr, b, x, *opts, FCGNO_FP64, info, (cudaStream_t)stream, nullptr, steps);
}

extern "C" fcgno_status fcgno_fp64_fma_rate(int blocks, int steps, double a, double c, double* out,
                                            uint64_t* fmas, void* stream) {
  if (blocks < 1 || blocks > (1 << 20) || steps < 1 || steps > (1 << 24) || !out || !fmas) {
    set_last_error("fcgno_fp64_fma_rate: blocks outside 1..2^20, steps outside 1..2^24, or null out/fmas");
    return FCGNO_EINVAL;
  }
  fp64_fma_rate_kernel<<<blocks, kRateThreads, 0, (cudaStream_t)stream>>>(steps, a, c, out);
  FCGNO_LAUNCHED();
  *fmas = (uint64_t)blocks * kRateThreads * kRateChains * (uint64_t)steps;
  return FCGNO_OK;
}

namespace fcgno {
// Device state of fcgno_solve_host kept between calls: the copies of k, b, x and the assembled
// operator (with its Krylov workspace and captured graphs) of the last shapes seen per device,
// so that repeated end-to-end solves of one shape re-assemble in place instead of allocating,
// assembling from scratch and capturing new graphs. Each entry has its own lock; a call that
// finds its entry in use by another thread works on temporary buffers instead.
struct HostSolveEntry {
  int dev = -1, N = 0, B = 0;
  double* dk = nullptr;
  double* db = nullptr;
  double* dx = nullptr;
  fcgno_op_t op = nullptr;
  uint64_t used = 0;
  std::mutex mu;
};
constexpr int kHostSolveEntries = 4;
static HostSolveEntry g_host_solve[kHostSolveEntries];
static std::mutex g_host_solve_mu;  // guards the entries' keys and the use counter
static uint64_t g_host_solve_clock = 0;

static void host_entry_free(HostSolveEntry& e) {
  if (e.op) fcgno_op_destroy(e.op);
  if (e.dk) cudaFree(e.dk);
  if (e.db) cudaFree(e.db);
  if (e.dx) cudaFree(e.dx);
  e.op = nullptr;
  e.dk = e.db = e.dx = nullptr;
  e.dev = -1;
  e.N = e.B = 0;
}

static fcgno_status host_solve_on(int N, int batch, double* dk, double* db, double* dx, fcgno_op_t* op_io,
                                  const double* k_host, const double* b_host, double* x_host, fcgno_model_t Bpc,
                                  const fcgno_solve_opts* opts, fcgno_prec prec, fcgno_solve_info* info,
                                  cudaStream_t st) {
  const size_t bytes = (size_t)N * N * batch * sizeof(double);
  if (cudaMemcpyAsync(dk, k_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(db, b_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dx, x_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    set_last_error("fcgno_solve_host: host-to-device copy failed");
    return FCGNO_ECUDA;
  }
  if (*op_io)
    FCGNO_TRY(fcgno_reassemble(*op_io, dk, st));
  else
    FCGNO_TRY(fcgno_assemble(N, batch, dk, st, op_io));
  FCGNO_TRY(fcgno_solve(*op_io, Bpc, db, dx, opts, prec, info, st));
  if (cudaMemcpyAsync(x_host, dx, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_last_error("fcgno_solve_host: device-to-host copy failed");
    return FCGNO_ECUDA;
  }
  return FCGNO_OK;
}
}  // namespace fcgno

extern "C" fcgno_status fcgno_solve_host(int N, int batch, const double* k_host, const double* b_host,
                                         double* x_host, fcgno_model_t Bpc, const fcgno_solve_opts* opts,
                                         fcgno_prec prec, fcgno_solve_info* info, void* stream) {
  if (N < 2 || batch < 1 || !k_host || !b_host || !x_host) {
    set_last_error("fcgno_solve_host: bad arguments");
    return FCGNO_EINVAL;
  }
  FCGNO_TRY(check_solve_args("fcgno_solve_host", N, Bpc, opts, prec));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)N * N * batch * sizeof(double);
  int dev = 0;
  FCGNO_CUDA_TRY(cudaGetDevice(&dev));
  // the cached entry of this shape (or the least recently used free one)
  HostSolveEntry* e = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_host_solve_mu);
    for (auto& c : g_host_solve)
      if (c.dev == dev && c.N == N && c.B == batch) e = &c;
    if (e && !e->mu.try_lock()) e = nullptr;
    if (!e) {
      HostSolveEntry* victim = nullptr;
      for (auto& c : g_host_solve) {
        if (!c.mu.try_lock()) continue;
        if (!victim || c.used < victim->used) {
          if (victim) victim->mu.unlock();
          victim = &c;
        } else {
          c.mu.unlock();
        }
      }
      e = victim;
      if (e && !(e->dev == dev && e->N == N && e->B == batch)) host_entry_free(*e);
    }
    if (e) e->used = ++g_host_solve_clock;
  }
  if (e) {
    std::lock_guard<std::mutex> hold(e->mu, std::adopt_lock);
    if (!e->dk) {
      if (cudaMalloc(&e->dk, bytes) != cudaSuccess || cudaMalloc(&e->db, bytes) != cudaSuccess ||
          cudaMalloc(&e->dx, bytes) != cudaSuccess) {
        cudaGetLastError();
        host_entry_free(*e);
        set_last_error("fcgno_solve_host: out of device memory");
        return FCGNO_ENOMEM;
      }
      e->dev = dev;
      e->N = N;
      e->B = batch;
    }
    const fcgno_status rc = host_solve_on(N, batch, e->dk, e->db, e->dx, &e->op, k_host, b_host, x_host, Bpc, opts,
                                          prec, info, st);
    if (rc != FCGNO_OK && rc != FCGNO_ETIMEOUT) host_entry_free(*e);
    return rc;
  }
  // every entry is in use by another thread: temporary buffers
  double *dk = nullptr, *db = nullptr, *dx = nullptr;
  if (cudaMallocAsync(&dk, bytes, st) != cudaSuccess || cudaMallocAsync(&db, bytes, st) != cudaSuccess ||
      cudaMallocAsync(&dx, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    if (dk) cudaFreeAsync(dk, st);
    if (db) cudaFreeAsync(db, st);
    set_last_error("fcgno_solve_host: out of device memory");
    return FCGNO_ENOMEM;
  }
  fcgno_op_t op = nullptr;
  const fcgno_status rc = host_solve_on(N, batch, dk, db, dx, &op, k_host, b_host, x_host, Bpc, opts, prec, info, st);
  if (op) fcgno_op_destroy(op);
  cudaFreeAsync(dk, st);
  cudaFreeAsync(db, st);
  cudaFreeAsync(dx, st);
  return rc;
}

extern "C" fcgno_status fcgno_solve_host_release(void) {
  using namespace fcgno;
  std::lock_guard<std::mutex> lk(g_host_solve_mu);
  for (auto& c : g_host_solve) {
    std::lock_guard<std::mutex> hold(c.mu);
    host_entry_free(c);
  }
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_krylov_harvest(fcgno_op_t A, const double* b, const double* x0,
                                             const double* u_star, int K, double* r_out, double* e_out,
                                             fcgno_solve_info* info, void* stream) {
  if (!A || !b || !x0 || !u_star || K < 1 || !r_out || !e_out) {
    set_last_error("fcgno_krylov_harvest: bad arguments");
    return FCGNO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = A->n * A->B * sizeof(double);
  double* u = nullptr;
  if (cudaMallocAsync(&u, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("fcgno_krylov_harvest: out of device memory");
    return FCGNO_ENOMEM;
  }
  fcgno_status rc = FCGNO_OK;
  if (cudaMemcpyAsync(u, x0, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    set_last_error("fcgno_krylov_harvest: copy failed");
    rc = FCGNO_ECUDA;
  } else {
    fcgno_solve_opts o{1e-13, 1, K, 0, K};  // converged instances keep their last iterate
    HarvestHook h{u_star, r_out, e_out};
    rc = solve_impl(A, nullptr, b, u, o, FCGNO_FP64, info, st, &h);
  }
  cudaFreeAsync(u, st);
  return rc;
}

// ------------------------------------ allocation-free solve ----------------------------
// Some callers cannot allocate device memory at solve time: code running under a fixed,
// pre-reserved memory budget, or inside a region where the CUDA allocator must not be
// entered. fcgno_solve_noalloc serves them for the identity preconditioner: its Krylov
// state lives in one file-scope device array of fixed size that every GPU loading this
// library holds until the process exits. All calls share that array.
namespace fcgno {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static void* g_noalloc_addr[64] = {};  // device address of the array, per device ordinal
static std::mutex g_noalloc_mu;         // guards g_noalloc_addr

// Device address of the scratch array for the current device. The first call on a device
// resolves it with cudaGetSymbolAddress (host code cannot use the symbol's own address);
// threads racing on that first call take the lock, so each device is resolved once.
static fcgno_status noalloc_scratch_address(void** out) {
  int dev = -1;
  FCGNO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_last_error("fcgno_solve_noalloc: device ordinal out of range");
    return FCGNO_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    FCGNO_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return FCGNO_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace fcgno

extern "C" fcgno_status fcgno_solve_noalloc(fcgno_op_t A, const double* b, double* x, const fcgno_solve_opts* opts,
                                            fcgno_solve_info* info, void* stream) {
  using namespace fcgno;
  if (!A || !b || !x) {
    set_last_error("fcgno_solve_noalloc: null operator, b or x");
    return FCGNO_EINVAL;
  }
  FCGNO_TRY(check_opts(opts));
  const fcgno_solve_opts& o = *opts;
  cudaStream_t st = (cudaStream_t)stream;
  const int slots = o.m_max + 1;
  const int B = A->B;
  const int tiles = (int)ceil_div(A->n, kTile);
  // carve the fixed array: r, P, S, per-instance scalars, partial sums, status words
  const size_t vec = A->n * (size_t)B * sizeof(double);
  size_t off[14];
  const size_t sizes[14] = {vec,
                            vec * slots,
                            vec * slots,
                            sizeof(double) * slots * B,
                            sizeof(double) * kMaxWindow * B,
                            sizeof(double) * B,
                            sizeof(double) * B,
                            sizeof(double) * B,
                            sizeof(double) * B,
                            sizeof(double) * (size_t)B * tiles * kParts,
                            sizeof(int) * B,
                            sizeof(int) * B,
                            sizeof(int),
                            sizeof(int)};
  size_t total = 0;
  for (int i = 0; i < 14; ++i) {
    off[i] = total;
    total += align256(sizes[i]);
  }
  if (total > kNoAllocScratchBytes) {
    set_last_error("fcgno_solve_noalloc: problem needs " + std::to_string(total) +
                   " bytes of solver scratch; the allocation-free solve is limited to " +
                   std::to_string(kNoAllocScratchBytes) + " bytes (8 MiB)");
    return FCGNO_EINVAL;
  }
  void* base_v = nullptr;
  FCGNO_TRY(noalloc_scratch_address(&base_v));
  unsigned char* base = (unsigned char*)base_v;
  State s;
  s.aE = A->aE;
  s.aN = A->aN;
  s.diag = A->diag;
  s.b = b;
  s.u = x;
  s.r = (double*)(base + off[0]);
  s.w = s.r;  // identity preconditioner: w_i = r_i
  s.P = (double*)(base + off[1]);
  s.S = (double*)(base + off[2]);
  s.ps = (double*)(base + off[3]);
  s.beta = (double*)(base + off[4]);
  s.alpha = (double*)(base + off[5]);
  s.r0 = (double*)(base + off[6]);
  s.rr = (double*)(base + off[7]);
  s.rms = (double*)(base + off[8]);
  s.part = (double*)(base + off[9]);
  s.status = (int*)(base + off[10]);
  s.iters = (int*)(base + off[11]);
  s.ndone = (int*)(base + off[12]);
  s.iter = (int*)(base + off[13]);
  IterArgs a{};
  a.N = A->N;
  a.B = B;
  a.n = A->n;
  a.tiles = tiles;
  a.nslots = slots;
  a.tol = o.tol;
  a.fixed = o.fixed_iters ? 1 : 0;
  const LoopShape L = loop_shape(A);
  FCGNO_TRY(prepare_fused(L));
  // the stopped-instance and iteration counters must start at zero: the array keeps the
  // previous call's data
  FCGNO_CUDA_TRY(cudaMemsetAsync(s.ndone, 0, sizeof(int), st));
  FCGNO_CUDA_TRY(cudaMemsetAsync(s.iter, 0, sizeof(int), st));
  init_kernel<<<dim3(a.tiles, B), kThreads, 0, st>>>(a, s);
  FCGNO_LAUNCHED();
  init_finalize_kernel<<<B, kThreads, 0, st>>>(a, s);
  FCGNO_LAUNCHED();
  const int check_every = std::max(1, o.check_every);
  int h_ndone = 0, since_check = 0, cur = check_every;
  for (int i = 0; i < o.max_iter; ++i) {
    FCGNO_TRY(launch_vector_step(a, s, L, st));
    if (++since_check >= cur || i + 1 == o.max_iter) {
      FCGNO_CUDA_TRY(cudaMemcpyAsync(&h_ndone, s.ndone, sizeof(int), cudaMemcpyDeviceToHost, st));
      FCGNO_CUDA_TRY(cudaStreamSynchronize(st));
      if (h_ndone >= B) break;
      since_check = 0;
      cur = B - h_ndone <= kTailRunning ? std::min(check_every, kTailReplay) : check_every;
    }
  }
  // per-instance results, copied through fixed-size host buffers
  constexpr int kChunk = 64;
  int hs[kChunk], hi[kChunk];
  double hrr[kChunk], hr0[kChunk];
  for (int b0 = 0; b0 < B; b0 += kChunk) {
    const int cnt = std::min(kChunk, B - b0);
    FCGNO_CUDA_TRY(cudaMemcpyAsync(hs, s.status + b0, sizeof(int) * cnt, cudaMemcpyDeviceToHost, st));
    FCGNO_CUDA_TRY(cudaMemcpyAsync(hi, s.iters + b0, sizeof(int) * cnt, cudaMemcpyDeviceToHost, st));
    FCGNO_CUDA_TRY(cudaMemcpyAsync(hrr, s.rr + b0, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    FCGNO_CUDA_TRY(cudaMemcpyAsync(hr0, s.r0 + b0, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    FCGNO_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) {
      for (int j = 0; j < cnt; ++j) {
        int stt = hs[j];
        if (stt == kRunning) stt = o.fixed_iters ? FCGNO_OK : FCGNO_ENOCONV;
        info[b0 + j].iters = hi[j];
        info[b0 + j].status = stt;
        info[b0 + j].r0norm = hr0[j];
        info[b0 + j].relres = hr0[j] > 0 ? std::sqrt(hrr[j]) / hr0[j] : 0.0;
      }
    }
  }
  return FCGNO_OK;
}

namespace fcgno {

// ------------------------------------ device-driven serving ----------------------------
// Admission and retirement of a bucket's slots at the start of every iteration, on the device.
// The request queue and the result ring are pinned host memory mapped into the device's address
// space: the host publishes requests by advancing req_tail (release), the device publishes
// results by writing each record's sequence number last (after a system-scope fence). Slot
// phases: 0 free, 1 solving, 2 retiring (this iteration), 3 admitted (this iteration).
struct ServeDev {
  int qcap, dcap, max_iter, grid;
  const fcgno_serve_request* req;       // [qcap] (mapped)
  const unsigned long long* req_tail;   // requests published by the host (mapped)
  unsigned long long* req_head_pub;     // requests taken by the device (mapped, for the host)
  fcgno_serve_result* res;              // [dcap] (mapped)
  const unsigned long long* res_head;   // results consumed by the host (mapped)
  unsigned long long* ctr;              // [2] requests taken, results published (device)
  fcgno_serve_request* slot_req;        // [B] each slot's request (device)
  int* phase;                           // [B]
  int* list;                            // [2][B] retiring slots, admitted slots
  int* count;                           // [2] their numbers
  double* x;                            // the bucket's iterates [B][n]
  double* b;                            // the bucket's right-hand sides [B][n]
  double* aE;
  double* aN;
  double* diag;
  double* logk;
  float* logk32;
  double* kinv;
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix count of `flag` over the block (1024 threads max) in thread order; *total
// receives the block's count. Contains two __syncthreads().
__device__ __forceinline__ int block_rank(bool flag, int* warp_counts, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) warp_counts[warp] = __popc(m);
  __syncthreads();
  int before = 0, tot = 0;
  for (int w = 0; w < nw; ++w) {
    if (w < warp) before += warp_counts[w];
    tot += warp_counts[w];
  }
  __syncthreads();
  *total = tot;
  return before + __popc(m & ((1u << lane) - 1u));
}

// (1) one block: lists the slots to retire (their solve stopped, and the result ring has room)
// and admits queued requests into free slots, both in slot order.
__global__ void __launch_bounds__(1024) serve_scan_kernel(ServeDev v, State s, int B) {
  __shared__ int wc[32];
  __shared__ unsigned long long avail_q, avail_r;
  if (threadIdx.x == 0) {
    const unsigned long long tail = ld_acquire_sys(v.req_tail);
    const unsigned long long head = v.ctr[0];
    avail_q = tail > head ? tail - head : 0ull;
    const unsigned long long consumed = ld_acquire_sys(v.res_head);
    const unsigned long long used = v.ctr[1] - consumed;
    avail_r = used < (unsigned long long)v.dcap ? (unsigned long long)v.dcap - used : 0ull;
  }
  __syncthreads();
  int nR = 0, nA = 0;
  for (int base = 0; base < B; base += blockDim.x) {
    const int slot = base + threadIdx.x;
    bool isR = false, isF = false;
    if (slot < B) {
      const int ph = v.phase[slot];
      isR = ph == 1 && (s.status[slot] != kRunning || s.iters[slot] >= v.max_iter);
      isF = ph == 0;
    }
    int totR, totF;
    const int rR = block_rank(isR, wc, &totR);
    const int rF = block_rank(isF, wc, &totF);
    if (isR && (unsigned long long)(nR + rR) < avail_r) {
      v.list[nR + rR] = slot;
      v.phase[slot] = 2;
      if (s.status[slot] == kRunning) s.status[slot] = FCGNO_ENOCONV;  // capped: stop it
    }
    if (isF && (unsigned long long)(nA + rF) < avail_q) {
      const unsigned long long idx = v.ctr[0] + (unsigned long long)(nA + rF);
      const volatile fcgno_serve_request* rq = v.req + idx % (unsigned long long)v.qcap;
      fcgno_serve_request r;
      r.k = rq->k;
      r.f = rq->f;
      r.x0 = rq->x0;
      r.x_out = rq->x_out;
      r.tag = rq->tag;
      v.slot_req[slot] = r;
      v.phase[slot] = 3;
      v.list[B + nA + rF] = slot;
    }
    nR = (int)min((unsigned long long)(nR + totR), avail_r);
    nA = (int)min((unsigned long long)(nA + totF), avail_q);
  }
  __syncthreads();  // every thread has read ctr[0]
  if (threadIdx.x == 0) {
    v.count[0] = nR;
    v.count[1] = nA;
    v.ctr[0] += (unsigned long long)nA;
    st_release_sys(v.req_head_pub, v.ctr[0]);
  }
}

// (2) retiring slots: iterate -> the request's x_out; admitted slots: operator assembled from
// the request's k, f and x0 copied in. The two lists hold different slots.
__global__ void __launch_bounds__(256) serve_move_kernel(ServeDev v, int N, size_t n, int B) {
  const int nR = v.count[0], nA = v.count[1];
  const size_t total = (size_t)(nR + nA) * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int which = (int)(idx / n);
    const size_t e = idx - (size_t)which * n;
    if (which < nR) {
      const int slot = v.list[which];
      v.slot_req[slot].x_out[e] = v.x[(size_t)slot * n + e];
    } else {
      const int slot = v.list[B + which - nR];
      const fcgno_serve_request& r = v.slot_req[slot];
      const size_t i = (size_t)slot * n + e;
      assemble_point(N, (int)e, r.k, i, v.aE, v.aN, v.diag, v.logk, v.logk32, v.kinv);
      v.b[i] = r.f[e];
      v.x[i] = r.x0[e];
    }
  }
}

// (3) admitted slots: r_0 = b - A x0 and the per-tile partial sums of ||r_0||^2 (as init_kernel)
__global__ void __launch_bounds__(kThreads) serve_init_kernel(ServeDev v, IterArgs a, State s) {
  __shared__ double scratch[32];
  const int nA = v.count[1];
  for (int job = blockIdx.x; job < nA * a.tiles; job += gridDim.x) {
    const int b = v.list[a.B + job / a.tiles], tile = job % a.tiles;
    const size_t off = (size_t)b * a.n;
    double acc[1] = {0.0};
    for (int j = 0; j < kEPT; ++j) {
      const size_t e = (size_t)tile * kTile + j * kThreads + threadIdx.x;
      if (e < a.n) {
        const int q = (int)(e / a.N), p = (int)(e - (size_t)q * a.N);
        const double* u = s.u + off;
        const double c = u[e];
        const double ue = (p < a.N - 1) ? u[e + 1] : 0.0;
        const double uw = (p > 0) ? u[e - 1] : 0.0;
        const double un = (q < a.N - 1) ? u[e + a.N] : 0.0;
        const double us = (q > 0) ? u[e - a.N] : 0.0;
        const double rv = s.b[off + e] - stencil_at(s, off + e, p, q, a.N, c, ue, uw, un, us);
        s.r[off + e] = rv;
        acc[0] = fma(rv, rv, acc[0]);
      }
    }
    const double tot = block_sum_lane<double, 1>(acc, 1, scratch);
    if (threadIdx.x == 0) s.part[((size_t)b * a.tiles + tile) * kParts] = tot;
    __syncthreads();
  }
}

// (4) one block: publishes the retiring slots' results (their x_out is written) and frees them;
// finishes the admitted slots (||r_0||, rms, iteration 0, running).
__global__ void __launch_bounds__(kThreads) serve_finish_kernel(ServeDev v, IterArgs a, State s) {
  __shared__ double scratch[32];
  const int nR = v.count[0], nA = v.count[1];
  for (int i = threadIdx.x; i < nR; i += blockDim.x) {
    const int slot = v.list[i];
    const unsigned long long seq = v.ctr[1] + (unsigned long long)i + 1ull;
    fcgno_serve_result* rec = v.res + (seq - 1ull) % (unsigned long long)v.dcap;
    rec->tag = v.slot_req[slot].tag;
    rec->status = s.status[slot];
    rec->iters = s.iters[slot];
    rec->relres = s.r0[slot] > 0.0 ? sqrt(s.rr[slot]) / s.r0[slot] : 0.0;
    __threadfence_system();
    st_release_sys(reinterpret_cast<unsigned long long*>(&rec->seq), seq);
    v.phase[slot] = 0;
  }
  for (int j = 0; j < nA; ++j) {
    const int b = v.list[a.B + j];
    const double rr = tile_totals<1>(a, s, b, 1, 0, scratch);
    if (threadIdx.x == 0) {
      s.rr[b] = rr;
      s.r0[b] = sqrt(rr);
      s.rms[b] = sqrt(rr / (double)a.n);
      s.iters[b] = 0;
      s.status[b] = rr == 0.0 ? FCGNO_OK : kRunning;
      v.phase[b] = 1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) v.ctr[1] += (unsigned long long)nR;
}

static fcgno_status launch_serve(const ServeDev& v, const IterArgs& a, const State& s, cudaStream_t cs) {
  serve_scan_kernel<<<1, 1024, 0, cs>>>(v, s, a.B);
  FCGNO_LAUNCHED();
  serve_move_kernel<<<v.grid, 256, 0, cs>>>(v, a.N, a.n, a.B);
  FCGNO_LAUNCHED();
  serve_init_kernel<<<v.grid, kThreads, 0, cs>>>(v, a, s);
  FCGNO_LAUNCHED();
  serve_finish_kernel<<<1, kThreads, 0, cs>>>(v, a, s);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

// Host side of a bucket's device-driven serving: the mapped queue and ring, the device arrays.
struct ServeRings {
  void* mapped = nullptr;    // one pinned, mapped allocation holding the pieces below
  fcgno_serve_request* req = nullptr;
  unsigned long long* req_tail = nullptr;  // written by the host
  unsigned long long* req_head = nullptr;  // written by the device
  fcgno_serve_result* res = nullptr;
  unsigned long long* res_head = nullptr;  // written by the host
  void* device = nullptr;    // one device allocation: counters, slot requests, phases, lists
  ServeDev dev{};
  unsigned long long host_tail = 0, host_head = 0;
  std::mutex mu;
};

}  // namespace fcgno

// ------------------------------------ serving buckets ----------------------------------
// A bucket keeps `capacity` same-size solves resident on the device (operator, iterate,
// right-hand side, Krylov state) and advances every active slot together. Slots are
// admitted and retired independently: every kernel derives the truncation window from the
// slot's own iteration count and skips slots whose status is not "running", so a slot's
// arithmetic does not depend on what the other slots are doing.
struct fcgno_bucket {
  fcgno_op* op = nullptr;
  fcgno_model* model = nullptr;
  fcgno_prec prec = FCGNO_BF16;
  double* x = nullptr;  // [capacity][n]
  double* b = nullptr;  // [capacity][n]
  fcgno::IterArgs a{};
  fcgno::State s{};
  fcgno::LoopShape L{};
  fcgno::LoopShape Ln{};  // narrow shape (few running slots)
  bool can_narrow = false;
  int G = 8;
  int max_iter = 1000;
  bool warmed = false;
  int* h_status = nullptr;  // pinned mirrors
  int* h_iters = nullptr;
  double* h_rr = nullptr;
  double* h_r0 = nullptr;
  int occupied = 0;         // slots admitted and not yet taken (host-driven mode)
  fcgno::ServeRings* srv = nullptr;  // device-driven serving (after fcgno_bucket_serve_enable)
};

extern "C" fcgno_status fcgno_bucket_create(int N, int capacity, fcgno_model_t model, fcgno_prec prec, int m_max,
                                            double tol, int max_iter, int iters_per_step, void* stream,
                                            fcgno_bucket_t* out) {
  using namespace fcgno;
  if (N < 2 || capacity < 1 || m_max < 1 || m_max > kMaxWindow || !(tol >= 0.0) || max_iter < 1 ||
      iters_per_step < 1 || !out || (model && N < 2 * model->desc.modes) || prec < FCGNO_FP64 ||
      prec > FCGNO_FP32) {
    set_last_error("fcgno_bucket_create: bad arguments");
    return FCGNO_EINVAL;
  }
  if (model && (prec == FCGNO_BF16 || prec == FCGNO_FP16) && !tc_shape_supported(N, model->desc)) {
    set_last_error(std::string("fcgno_bucket_create: ") + tc_shape_rule());
    return FCGNO_EINVAL;
  }
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  fcgno_bucket* k = new fcgno_bucket();
  fcgno_op* op = new fcgno_op();
  op->N = N;
  op->B = capacity;
  op->n = (size_t)N * N;
  k->op = op;
  k->model = model;
  k->prec = prec;
  k->G = iters_per_step;
  k->max_iter = max_iter;
  const size_t vec = op->n * capacity * sizeof(double);
  bool ok = cudaMalloc(&op->aE, vec) == cudaSuccess && cudaMalloc(&op->aN, vec) == cudaSuccess &&
            cudaMalloc(&op->diag, vec) == cudaSuccess && cudaMalloc(&op->logk, vec) == cudaSuccess &&
            cudaMalloc(&op->logk32, vec / 2) == cudaSuccess && cudaMalloc(&op->kinv, vec) == cudaSuccess &&
            cudaMalloc(&k->x, vec) == cudaSuccess &&
            cudaMalloc(&k->b, vec) == cudaSuccess &&
            cudaMallocHost(&k->h_status, sizeof(int) * capacity) == cudaSuccess &&
            cudaMallocHost(&k->h_iters, sizeof(int) * capacity) == cudaSuccess &&
            cudaMallocHost(&k->h_rr, sizeof(double) * capacity) == cudaSuccess &&
            cudaMallocHost(&k->h_r0, sizeof(double) * capacity) == cudaSuccess;
  fcgno_status rc = ok ? ensure_ws(op, m_max + 1) : FCGNO_ENOMEM;
  if (rc != FCGNO_OK) {
    cudaGetLastError();
    fcgno_bucket_destroy(k);
    set_last_error("fcgno_bucket_create: out of memory");
    return rc;
  }
  // Everything after the allocations fails through one path that destroys the bucket (and
  // its operator, workspace and pinned mirrors).
  auto setup = [&]() -> fcgno_status {
    // unused slots: neutral operator values, status "stopped" so that every kernel skips them
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->aE, 0, vec, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->aN, 0, vec, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->logk, 0, vec, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->logk32, 0, vec / 2, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->kinv, 0, vec, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(k->x, 0, vec, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(k->b, 0, vec, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->ws.r, 0, vec, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->ws.rms, 0, sizeof(double) * capacity, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->ws.iters, 0, sizeof(int) * capacity, st));
    std::vector<int> stopped(capacity, FCGNO_OK);
    FCGNO_CUDA_TRY(
        cudaMemcpyAsync(op->ws.status, stopped.data(), sizeof(int) * capacity, cudaMemcpyHostToDevice, st));
    FCGNO_CUDA_TRY(cudaMemsetAsync(op->diag, 0, vec, st));
    FCGNO_CUDA_TRY(cudaStreamSynchronize(st));
    SolverWorkspace& w = op->ws;
    const bool identity = (model == nullptr);
    k->s = make_state(op, k->b, k->x, identity ? w.r : w.w);
    k->a.N = N;
    k->a.B = capacity;
    k->a.n = op->n;
    k->a.tiles = (int)ceil_div(op->n, kTile);
    k->a.nslots = m_max + 1;
    k->a.tol = tol;
    k->a.fixed = 0;
    k->L = loop_shape(op);
    k->Ln = loop_shape(op, true);
    FCGNO_TRY(prepare_fused(k->L));
    FCGNO_TRY(prepare_fused(k->Ln));
    const bool tc = model && (prec == FCGNO_BF16 || prec == FCGNO_FP16);
    k->can_narrow = (tc && tc_has_narrow(N, model->desc)) || k->Ln.CL != k->L.CL;
    return FCGNO_OK;
  };
  rc = setup();
  if (rc != FCGNO_OK) {
    const std::string why = fcgno_last_error();
    cudaGetLastError();
    fcgno_bucket_destroy(k);
    set_last_error("fcgno_bucket_create: " + why);
    return rc;
  }
  *out = k;
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_bucket_admit(fcgno_bucket_t k, int slot, const double* kcoef, const double* f,
                                           const double* x0, void* stream) {
  using namespace fcgno;
  if (!k || slot < 0 || slot >= k->op->B || !kcoef || !f || !x0 || k->srv) {
    set_last_error(k && k->srv ? "fcgno_bucket_admit: the bucket serves from its device queue"
                               : "fcgno_bucket_admit: bad arguments");
    return FCGNO_EINVAL;
  }
  ++k->occupied;
  cudaStream_t st = (cudaStream_t)stream;
  fcgno_op* op = k->op;
  const size_t n = op->n, off = (size_t)slot * n;
  // the slot's operator, right-hand side and initial guess
  FCGNO_TRY(launch_assemble(op, off, n, kcoef, st));
  FCGNO_CUDA_TRY(cudaMemcpyAsync(k->b + off, f, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  FCGNO_CUDA_TRY(cudaMemcpyAsync(k->x + off, x0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  // r_0, ||r_0||, status "running", iteration 0 for this slot only
  IterArgs a1 = k->a;
  a1.B = 1;
  State s1 = k->s;
  s1.aE += off;
  s1.aN += off;
  s1.diag += off;
  s1.b += off;
  s1.u += off;
  s1.r += off;
  s1.part += (size_t)slot * a1.tiles * kParts;
  s1.rr += slot;
  s1.r0 += slot;
  s1.rms += slot;
  s1.status += slot;
  s1.iters += slot;
  init_kernel<<<dim3(a1.tiles, 1), kThreads, 0, st>>>(a1, s1);
  FCGNO_LAUNCHED();
  init_finalize_kernel<<<1, kThreads, 0, st>>>(a1, s1);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_bucket_step(fcgno_bucket_t k, void* stream) {
  using namespace fcgno;
  if (!k) {
    set_last_error("fcgno_bucket_step: null bucket");
    return FCGNO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  SolverWorkspace& w = k->op->ws;
  FCGNO_CUDA_TRY(cudaEventRecord(w.ev_in, st));
  FCGNO_CUDA_TRY(cudaStreamWaitEvent(w.cs, w.ev_in, 0));
  const ServeDev* sv = k->srv ? &k->srv->dev : nullptr;
  // an upper bound on the running slots, known on the host: requests enqueued and not yet
  // collected (device-driven) or slots admitted and not yet taken; few running slots take the
  // narrow launch shapes (shorter serial chains), as a solve does
  long long bound = k->occupied;
  if (k->srv) {
    std::lock_guard<std::mutex> lk(k->srv->mu);
    bound = (long long)(k->srv->host_tail - k->srv->host_head);
  }
  const int mode = launch_shape_mode();
  const bool narrow = mode == 2 || (mode == 0 && k->can_narrow && bound <= kNarrowRunning);
  const LoopShape& L = narrow ? k->Ln : k->L;
  if (!k->warmed || !graphs_enabled() || k->G == 1) {
    // first step eagerly (lazily allocated buffers exist before any capture)
    for (int i = 0; i < k->G; ++i)
      FCGNO_TRY(launch_iteration(k->op, k->model, k->prec, k->a, k->s, L, w.cs, 0, narrow, sv));
    k->warmed = true;
  } else {
    FCGNO_TRY(ensure_graph(k->op, k->model, k->prec, k->a, k->s, L, k->b, k->x, k->G, 0, narrow, sv));
    FCGNO_CUDA_TRY(cudaGraphLaunch(w.graph[narrow ? 1 : 0].exec, w.cs));
    g_launches.fetch_add(w.graph[narrow ? 1 : 0].kernels, std::memory_order_relaxed);
  }
  FCGNO_CUDA_TRY(cudaEventRecord(w.ev_out, w.cs));
  FCGNO_CUDA_TRY(cudaStreamWaitEvent(st, w.ev_out, 0));
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_bucket_poll(fcgno_bucket_t k, int32_t* status, int32_t* iters, double* relres,
                                          void* stream) {
  using namespace fcgno;
  if (!k || !status || !iters || !relres) {
    set_last_error("fcgno_bucket_poll: bad arguments");
    return FCGNO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  SolverWorkspace& w = k->op->ws;
  const int B = k->op->B;
  FCGNO_CUDA_TRY(cudaMemcpyAsync(k->h_status, w.status, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  FCGNO_CUDA_TRY(cudaMemcpyAsync(k->h_iters, w.iters, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
  FCGNO_CUDA_TRY(cudaMemcpyAsync(k->h_rr, w.rr, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  FCGNO_CUDA_TRY(cudaMemcpyAsync(k->h_r0, w.r0, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
  FCGNO_CUDA_TRY(cudaStreamSynchronize(st));
  FCGNO_TRY(tc_take_timeout(k->op, st));
  for (int i = 0; i < B; ++i) {
    int stt = k->h_status[i];
    if (stt == kRunning && k->h_iters[i] >= k->max_iter) stt = FCGNO_ENOCONV;
    status[i] = stt;
    iters[i] = k->h_iters[i];
    relres[i] = k->h_r0[i] > 0 ? std::sqrt(k->h_rr[i]) / k->h_r0[i] : 0.0;
  }
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_bucket_take(fcgno_bucket_t k, int slot, double* x_out, void* stream) {
  using namespace fcgno;
  if (!k || slot < 0 || slot >= k->op->B || k->srv) {
    set_last_error(k && k->srv ? "fcgno_bucket_take: the bucket serves from its device queue"
                               : "fcgno_bucket_take: bad arguments");
    return FCGNO_EINVAL;
  }
  if (k->occupied > 0) --k->occupied;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = k->op->n, off = (size_t)slot * n;
  if (x_out) FCGNO_CUDA_TRY(cudaMemcpyAsync(x_out, k->x + off, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  // stop the slot (a capped slot is still "running" on the device)
  const int stopped = FCGNO_ENOCONV;
  int cur = 0;
  FCGNO_CUDA_TRY(cudaMemcpyAsync(&cur, k->op->ws.status + slot, sizeof(int), cudaMemcpyDeviceToHost, st));
  FCGNO_CUDA_TRY(cudaStreamSynchronize(st));
  if (cur == kRunning)
    FCGNO_CUDA_TRY(cudaMemcpyAsync(k->op->ws.status + slot, &stopped, sizeof(int), cudaMemcpyHostToDevice, st));
  FCGNO_CUDA_TRY(cudaStreamSynchronize(st));
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_bucket_serve_enable(fcgno_bucket_t k, int queue_capacity, int result_capacity) {
  using namespace fcgno;
  if (!k || queue_capacity < 1 || result_capacity < 1 || k->srv || k->occupied != 0) {
    set_last_error(!k ? "fcgno_bucket_serve_enable: null bucket"
                      : (k->srv ? "fcgno_bucket_serve_enable: already enabled"
                                : (k->occupied ? "fcgno_bucket_serve_enable: slots still admitted (take them first)"
                                               : "fcgno_bucket_serve_enable: capacities must be >= 1")));
    return FCGNO_EINVAL;
  }
  const int B = k->op->B;
  ServeRings* r = new ServeRings();
  const size_t q = (size_t)queue_capacity, d = (size_t)result_capacity;
  // mapped: requests | results | 3 counters (each piece 64-byte aligned)
  auto al = [](size_t x) { return (x + 63) & ~(size_t)63; };
  const size_t o_res = al(q * sizeof(fcgno_serve_request)), o_ctr = o_res + al(d * sizeof(fcgno_serve_result));
  const size_t mapped_bytes = o_ctr + 3 * 64;
  // device: counters [2] | count [2] | slot requests [B] | phase [B] | lists [2B]
  const size_t o_cnt = 64, o_sreq = 128, o_ph = o_sreq + al((size_t)B * sizeof(fcgno_serve_request));
  const size_t o_list = o_ph + al((size_t)B * sizeof(int)), dev_bytes = o_list + al((size_t)2 * B * sizeof(int));
  void* mdev = nullptr;
  int sms = 0, devno = 0;
  cudaError_t e = cudaHostAlloc(&r->mapped, mapped_bytes, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&mdev, r->mapped, 0);
  if (e == cudaSuccess) e = cudaMalloc(&r->device, dev_bytes);
  if (e == cudaSuccess) e = cudaGetDevice(&devno);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devno);
  if (e == cudaSuccess) e = cudaMemset(r->device, 0, dev_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (r->mapped) cudaFreeHost(r->mapped);
    if (r->device) cudaFree(r->device);
    delete r;
    set_last_error(std::string("fcgno_bucket_serve_enable: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FCGNO_ENOMEM : FCGNO_ECUDA;
  }
  std::memset(r->mapped, 0, mapped_bytes);
  unsigned char* hm = (unsigned char*)r->mapped;
  unsigned char* dm = (unsigned char*)mdev;
  unsigned char* dd = (unsigned char*)r->device;
  r->req = (fcgno_serve_request*)hm;
  r->res = (fcgno_serve_result*)(hm + o_res);
  r->req_tail = (unsigned long long*)(hm + o_ctr);
  r->req_head = (unsigned long long*)(hm + o_ctr + 64);
  r->res_head = (unsigned long long*)(hm + o_ctr + 128);
  ServeDev& v = r->dev;
  v.qcap = queue_capacity;
  v.dcap = result_capacity;
  v.max_iter = k->max_iter;
  v.grid = std::max(1, sms) * 8;
  v.req = (const fcgno_serve_request*)dm;
  v.res = (fcgno_serve_result*)(dm + o_res);
  v.req_tail = (const unsigned long long*)(dm + o_ctr);
  v.req_head_pub = (unsigned long long*)(dm + o_ctr + 64);
  v.res_head = (const unsigned long long*)(dm + o_ctr + 128);
  v.ctr = (unsigned long long*)dd;
  v.count = (int*)(dd + o_cnt);
  v.slot_req = (fcgno_serve_request*)(dd + o_sreq);
  v.phase = (int*)(dd + o_ph);
  v.list = (int*)(dd + o_list);
  fcgno_op* op = k->op;
  v.x = k->x;
  v.b = k->b;
  v.aE = op->aE;
  v.aN = op->aN;
  v.diag = op->diag;
  v.logk = op->logk;
  v.logk32 = op->logk32;
  v.kinv = op->kinv;
  k->srv = r;
  drop_graph(op->ws);  // the next step captures the admission and retirement kernels too
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_bucket_enqueue(fcgno_bucket_t k, const fcgno_serve_request* req) {
  using namespace fcgno;
  if (!k || !req || !k->srv || !req->k || !req->f || !req->x0 || !req->x_out) {
    set_last_error("fcgno_bucket_enqueue: null argument or a bucket without fcgno_bucket_serve_enable");
    return FCGNO_EINVAL;
  }
  ServeRings& r = *k->srv;
  std::lock_guard<std::mutex> lk(r.mu);
  const unsigned long long taken = __atomic_load_n(r.req_head, __ATOMIC_ACQUIRE);
  if (r.host_tail - taken >= (unsigned long long)r.dev.qcap) {
    set_last_error("fcgno_bucket_enqueue: queue full");
    return FCGNO_ENOMEM;
  }
  r.req[r.host_tail % (unsigned long long)r.dev.qcap] = *req;
  ++r.host_tail;
  __atomic_store_n(r.req_tail, r.host_tail, __ATOMIC_RELEASE);  // publishes the descriptor
  return FCGNO_OK;
}

extern "C" int fcgno_bucket_results(fcgno_bucket_t k, fcgno_serve_result* out, int max) {
  using namespace fcgno;
  if (!k || !out || !k->srv || max < 0) return -1;
  ServeRings& r = *k->srv;
  std::lock_guard<std::mutex> lk(r.mu);
  int n = 0;
  while (n < max) {
    fcgno_serve_result* rec = r.res + r.host_head % (unsigned long long)r.dev.dcap;
    const unsigned long long seq = __atomic_load_n(reinterpret_cast<unsigned long long*>(&rec->seq), __ATOMIC_ACQUIRE);
    if (seq != r.host_head + 1) break;
    out[n++] = *rec;
    ++r.host_head;
  }
  if (n) __atomic_store_n(r.res_head, r.host_head, __ATOMIC_RELEASE);  // frees the records
  return n;
}

extern "C" fcgno_status fcgno_bucket_destroy(fcgno_bucket_t k) {
  if (!k) return FCGNO_OK;
  if (k->srv) {
    cudaDeviceSynchronize();  // no step may still read the mapped queue
    if (k->srv->mapped) cudaFreeHost(k->srv->mapped);
    if (k->srv->device) cudaFree(k->srv->device);
    delete k->srv;
    k->srv = nullptr;
  }
  if (k->op) fcgno_op_destroy(k->op);
  if (k->x) cudaFree(k->x);
  if (k->b) cudaFree(k->b);
  if (k->h_status) cudaFreeHost(k->h_status);
  if (k->h_iters) cudaFreeHost(k->h_iters);
  if (k->h_rr) cudaFreeHost(k->h_rr);
  if (k->h_r0) cudaFreeHost(k->h_r0);
  delete k;
  return FCGNO_OK;
}
