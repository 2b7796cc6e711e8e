// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstddef>
#include <atomic>
#include <string>
#include <vector>

#include "../../include/fcgno.h"

namespace fcgno {

// ---------------------------------------------------------------------------------------
// Error handling and launch accounting
// ---------------------------------------------------------------------------------------
void set_last_error(const std::string& msg);
extern std::atomic<uint64_t> g_launches;

#define FCGNO_CUDA_TRY(call)                                                                 \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      ::fcgno::set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));           \
      cudaGetLastError(); /* clear a non-sticky error so later checks do not see it */      \
      return FCGNO_ECUDA;                                                                    \
    }                                                                                        \
  } while (0)

// Records a launch of one of this library's kernels and checks the launch itself.
#define FCGNO_LAUNCHED()                                                                     \
  do {                                                                                       \
    ::fcgno::g_launches.fetch_add(1, std::memory_order_relaxed);                             \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess) {                                                                 \
      ::fcgno::set_last_error(std::string("kernel launch: ") + cudaGetErrorString(e_));      \
      return FCGNO_ECUDA;                                                                    \
    }                                                                                        \
  } while (0)

#define FCGNO_TRY(call)                                                                      \
  do {                                                                                       \
    fcgno_status s_ = (call);                                                                \
    if (s_ != FCGNO_OK) return s_;                                                           \
  } while (0)

// Kernel tracing: when a kernel family is selected with fcgno_trace_set, its launch sites
// bracket the launch with a pair of CUDA events on the launch stream.
bool trace_enabled(const char* family);
void trace_begin(const char* family, cudaStream_t st);
void trace_end(const char* family, cudaStream_t st);
// While a CUDA graph is being captured, traced launches become event-record nodes; their
// event pairs go to `list`, and trace_accumulate adds their durations after each replay.
using EventPairs = std::vector<std::pair<cudaEvent_t, cudaEvent_t>>;
void trace_capture_begin(EventPairs* list);
void trace_capture_end();
void trace_accumulate(const EventPairs& pairs);
void trace_release(EventPairs& pairs);
uint64_t trace_generation();  // changes whenever the traced family changes
struct TraceScope {
  const char* fam;
  cudaStream_t st;
  bool on;
  TraceScope(const char* f, cudaStream_t s) : fam(f), st(s), on(trace_enabled(f)) {
    if (on) trace_begin(fam, st);
  }
  ~TraceScope() {
    if (on) trace_end(fam, st);
  }
};

// Programmatic dependent launch. The kernels of one FCG-NO iteration form a chain on one
// stream, and each link is launched so that it may start while its predecessor still runs:
// its set-up (shared and tensor memory, barriers, copies of constant tables and of data
// written two or more kernels earlier) overlaps the predecessor's tail. Rules kept by every
// chained kernel:
//  - pdl_wait() comes before any access to global memory that the predecessor writes, and
//    before any write to global memory that the predecessor reads;
//  - pdl_trigger() comes only after pdl_wait(), so that when a kernel starts, the kernel two
//    links back has completed and its writes are visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches `kernel` as a chained link (programmatic stream serialization) on `st`.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Per-instance solver status codes kept on the device (negative = still iterating).
// Launches `kernel` as a chained link whose CTAs form clusters of `cluster_x` x 1 x 1.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                          cudaStream_t st, int cluster_x, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = cluster_x;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

constexpr int kRunning = -1;
constexpr int kMaxWindow = 8;  // largest m_max supported

// ---------------------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------------------
// A captured CUDA graph of several solver iterations and the parameters baked into it.
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;  // kernel nodes per replay
  uint64_t trace_gen = 0;
  const void* model = nullptr;
  uint64_t model_gen = 0;
  int prec = -1, nslots = 0, fixed = 0, G = 0, jacobi = 0;
  double tol = 0.0;
  const void* b = nullptr;
  const void* x = nullptr;
  const void* serve = nullptr;  // device-driven serving hooks captured in the graph (or none)
  EventPairs traced;
};

struct SolverWorkspace {
  int cap_B = 0, cap_n = 0, cap_slots = 0, cap_tiles = 0;
  cudaStream_t cs = nullptr;     // internal stream (graph capture needs a non-default stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  IterGraph graph[4];       // replayed iterations: [0] wide, [1] narrow 16-bit preconditioner launches;
                            // [2], [3] the same, shorter, for the tail of a batch
  int* iter = nullptr;      // [1] device iteration counter
  double* r = nullptr;      // [B][n]
  double* w = nullptr;      // [B][n]  preconditioned residual
  double* wt = nullptr;     // [B][n]  Jacobi sweep scratch
  double* inv_diag = nullptr;  // [B][n] 1 / diag (Jacobi)
  double* P = nullptr;      // [slots][B][n] directions p_k
  double* S = nullptr;      // [slots][B][n] A p_k
  double* ps = nullptr;     // [slots][B]    (p_k, s_k)
  double* beta = nullptr;   // [B][kMaxWindow]
  double* alpha = nullptr;  // [B]
  double* r0 = nullptr;     // [B] ||r_0||
  double* rr = nullptr;     // [B] ||r_i||^2
  double* rms = nullptr;    // [B] sqrt(||r_i||^2 / n)
  double* part = nullptr;   // [B][tiles][kParts] partial sums
  int* status = nullptr;    // [B]
  int* iters = nullptr;     // [B]
  int* ndone = nullptr;     // [1] count of stopped instances
};

}  // namespace fcgno

namespace fcgno {
struct TcActs;  // per-operator activations of the tensor-core preconditioner
}  // namespace fcgno

struct fcgno_op {
  int N = 0, B = 0;
  size_t n = 0;
  double* aE = nullptr;    // [B][n] east-face coefficient / h^2 (boundary face at p = N-1)
  double* aN = nullptr;    // [B][n] north-face coefficient / h^2 (boundary face at q = N-1)
  double* diag = nullptr;  // [B][n] sum of the four face coefficients / h^2
  double* logk = nullptr;  // [B][n]
  float* logk32 = nullptr; // [B][n] (input of the 16-bit preconditioner)
  double* kinv = nullptr;  // [B][n] 1 / k (output scale of models with output_scale 1)
  fcgno::SolverWorkspace ws;
  // Activations of the 16-bit preconditioner applied to this operator's batch. They belong to
  // the operator, not the model, so that solves of different operators with one model may
  // run concurrently on different streams (a cache: allocated on first use).
  mutable fcgno::TcActs* tc_acts = nullptr;
};

namespace fcgno {

struct NoWorkspace;  // activations of the preconditioner (defined per implementation)
struct TcModel;      // tensor-core copies of the weights

}  // namespace fcgno

struct fcgno_model {
  fcgno_model_desc desc{};
  const float* w32 = nullptr;   // caller's FP32 master blob (device)
  double* w64 = nullptr;        // FP64 copy of the blob (device)
  size_t count = 0;             // floats in the blob
  fcgno::NoWorkspace* ws = nullptr;
  fcgno::TcModel* tc = nullptr;
  uint64_t gen = 0;             // bumped whenever a derived device buffer is (re)allocated
  int train_recompute = 0;      // 0: recompute pre-activations above a size threshold; 1: always; 2: never
};

namespace fcgno {

// Blob offsets (in elements) -- same order as documented in fcgno.h.
struct BlobLayout {
  size_t lift_w, lift_b, proj1_w, proj1_b, proj2_w, proj2_b, total;
  size_t w[16], b[16], r[16];
};
BlobLayout blob_layout(const fcgno_model_desc& d);

// Assembly of grid point x of one instance (Eq. (1)-(2), 5-point finite volumes): from that
// instance's k ([N][N]) it writes, at element i of the operator's arrays, the east and north
// face coefficients (harmonic mean of the two nodes' k for an interior face, k of the node for a
// boundary face), the diagonal (sum of the four faces), all scaled by 1/h^2, log k (FP64 and
// FP32) and 1/k. Each interior face is formed with the (lower node, upper node) argument order,
// so that the coupling seen from both sides is bit-identical and A is exactly symmetric.
__device__ __forceinline__ double harmonic_mean(double a, double b) { return 2.0 * a * b / (a + b); }
__device__ __forceinline__ void assemble_point(int N, int x, const double* __restrict__ kb, size_t i,
                                               double* __restrict__ aE, double* __restrict__ aN,
                                               double* __restrict__ diag, double* __restrict__ logk,
                                               float* __restrict__ logk32, double* __restrict__ kinv) {
  const int q = x / N, p = x - q * N;
  const double kP = kb[x];
  const double inv_h2 = (double)(N + 1) * (double)(N + 1);
  const double e = (p < N - 1) ? harmonic_mean(kP, kb[x + 1]) : kP;
  const double w = (p > 0) ? harmonic_mean(kb[x - 1], kP) : kP;
  const double nn = (q < N - 1) ? harmonic_mean(kP, kb[x + N]) : kP;
  const double s = (q > 0) ? harmonic_mean(kb[x - N], kP) : kP;
  aE[i] = e * inv_h2;
  aN[i] = nn * inv_h2;
  diag[i] = (e + w + nn + s) * inv_h2;
  const double lk = log(kP);
  logk[i] = lk;
  logk32[i] = (float)lk;
  kinv[i] = 1.0 / kP;
}

// Face coefficients, diagonal, log k and 1/k of `total` grid points (all instances or one slot)
// into the operator's arrays starting at element `off`.
fcgno_status launch_assemble(const fcgno_op* op, size_t off, size_t total, const double* k, cudaStream_t st);
// Stencil matvec y = A x for all instances (FP64).
fcgno_status launch_apply_A(const fcgno_op* op, const double* x, double* y, cudaStream_t st);

// Preconditioner entry points implemented by the CUDA-core (SIMT) and tensor-core paths.
// rms: [B] per-instance rms of r (device); active: [B] status array (nullptr = all
// active; an instance is skipped when active[b] >= 0).
fcgno_status no_apply_simt(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms,
                           const int* active, double* z, bool fp64, cudaStream_t st);
// narrow: launch the synthesis with narrower grid-column chunks (more blocks per instance,
// shorter serial chains), for launches in which few instances are still active.
fcgno_status no_apply_tc(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms,
                         const int* active, double* z, bool fp16, cudaStream_t st, bool narrow = false);
// Whether the narrow launch shape differs from the wide one for this grid and model.
bool tc_has_narrow(int N, const fcgno_model_desc& d);
// Launch-shape policy set by fcgno_set_launch_shape: 0 automatic, 1 always wide, 2 always narrow.
int launch_shape_mode();
// Whether the 16-bit (tensor-core) preconditioner supports model shape d on an N x N grid,
// and the rule in words (for error messages). Host-only.
bool tc_shape_supported(int N, const fcgno_model_desc& d);
const char* tc_shape_rule();
// Device bytes of the buffers each path allocates for a batch of B on an N x N grid (the
// sizes the allocating code uses): tensor-core activations per operator, CUDA-core buffers
// per model, the solver workspace per operator (slots = m_max + 1) and the assembled operator.
size_t tc_acts_bytes(int N, int B, const fcgno_model_desc& d);
size_t simt_buffers_bytes(int N, int B, const fcgno_model_desc& d, bool fp64);
size_t solver_ws_bytes(size_t n, int B, int slots);
size_t operator_bytes(size_t n, int B);
fcgno_status tc_model_sync(fcgno_model* m, cudaStream_t st);
void tc_model_free(fcgno_model* m);
void tc_acts_free(fcgno_op* op);
// Reads and clears the operator's tensor-core timeout flag (synchronises `st`): FCGNO_ETIMEOUT
// if a kernel of the 16-bit preconditioner gave up one of its bounded waits since the last call.
fcgno_status tc_take_timeout(const fcgno_op* op, cudaStream_t st);
// Failure-detection self-test of the bounded wait (see fcgno_wait_selftest).
fcgno_status tc_wait_probe(const fcgno_op* op, uint64_t limit_ns, cudaStream_t st);
void no_workspace_free(fcgno_model* m);

// Per-instance rms of r: rms[b] = sqrt(mean(r_b^2)).
fcgno_status launch_rms(const double* r, int B, size_t n, double* rms, cudaStream_t st);

// Training: energy-norm loss of Eq. (11), or (l2) the 2-norm ablation loss. prec: FCGNO_FP32,
// FCGNO_FP64 (CUDA cores throughout) or FCGNO_BF16 (the Fourier layers forward and backward
// on the tensor cores, the rest on CUDA cores in FP32).
fcgno_status train_step_simt(fcgno_model* m, fcgno_op* op, const double* r, const double* e,
                             float* loss, float* grad, fcgno_prec prec, bool l2, cudaStream_t st);
// The FP64 step with its loss and gradient stored in FP64 (fcgno_train_step_f64).
fcgno_status train_step_f64(fcgno_model* m, fcgno_op* op, const double* r, const double* e,
                            double* loss, double* grad, bool l2, cudaStream_t st);

// Pieces of the BF16 training step (tensor-core path; wide launch shape, every instance active).
// begin: weight images (forward and transposed) from the current master blob, forward and
// adjoint tables, activation and training buffers. forward: encoder and Fourier layers with the
// backward's saves; cx[l] (FP32 [B][mode][C] complex) receives layer l's analysis output.
// to_f32: saved layer input `which` (0..L), or the current input gradient (which = -1), as FP32
// [B][N][N][C]. act_bwd: the pre-activation gradient of layer l from the gradient of its output
// (gv32, FP32 [B][N][N][C]; null: the one the previous layer_bwd left), into gh32 and the
// tile-major copy layer_bwd reads. layer_bwd: adjoint analysis (kept: gspec), adjoint mixing and
// adjoint synthesis of layer l, leaving the gradient of its input.
fcgno_status tc_train_begin(fcgno_model* m, const fcgno_op* op, cudaStream_t st);
fcgno_status tc_train_forward(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms,
                              float* const* cx, cudaStream_t st);
fcgno_status tc_train_to_f32(const fcgno_model* m, const fcgno_op* op, int which, float* out, cudaStream_t st);
fcgno_status tc_train_act_bwd(const fcgno_model* m, const fcgno_op* op, int l, const float* gv32, float* gh32,
                              cudaStream_t st);
fcgno_status tc_train_layer_bwd(fcgno_model* m, const fcgno_op* op, int l, cudaStream_t st);
// recompute: with activation checkpointing (fcgno_model_set_train_recompute), rebuilds layer l's
// pre-activation from its kept input before act_bwd reads it (no-op otherwise).
fcgno_status tc_train_recompute_layer(fcgno_model* m, const fcgno_op* op, int l, cudaStream_t st);
bool tc_train_recompute(const fcgno_model* m, const fcgno_op* op);
const float* tc_train_gspec(const fcgno_op* op);
size_t tc_train_bytes(int N, int B, const fcgno_model_desc& d, bool recompute);

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block reduction of NV values per thread; the result is valid in every
// thread. scratch must hold 32*NV entries of T. Contains __syncthreads().
template <typename T, int NV>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) scratch[wid * NV + j] = v[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    T s = 0;
    for (int w = 0; w < nw; ++w) s += scratch[w * NV + j];
    v[j] = s;
  }
  __syncthreads();
}

// Fixed-order block reduction of the first `count` (<= NV) values of every thread. Returns the
// block total of value j in thread j (j < count) and 0 elsewhere; only those entries are
// reduced, and one thread per entry adds up the warp partials. scratch must hold 32*NV
// entries of T. Contains __syncthreads().
template <typename T, int NV>
__device__ __forceinline__ T block_sum_lane(T (&v)[NV], int count, T* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j)
    if (j < count) v[j] = warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < count) scratch[wid * NV + j] = v[j];
  }
  __syncthreads();
  T s = 0;
  if ((int)threadIdx.x < count)
    for (int w = 0; w < nw; ++w) s += scratch[w * NV + threadIdx.x];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double gelu_d(double x) { return 0.5 * x * (1.0 + erf(x * 0.70710678118654752440)); }
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752440f)); }
// d/dx GELU(x) = Phi(x) + x phi(x)
__device__ __forceinline__ double gelu_grad_d(double x) {
  return 0.5 * (1.0 + erf(x * 0.70710678118654752440)) + x * 0.39894228040143267794 * exp(-0.5 * x * x);
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752440f)) + x * 0.39894228040143267794f * expf(-0.5f * x * x);
}

}  // namespace fcgno
