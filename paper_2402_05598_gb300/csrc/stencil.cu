// Stencil assembly and matrix-free application of the discretised Eq. (1)-(2).
//
// -div(k grad u) = f on (0,1)^2, u = 0 on the boundary, 5-point finite volume on the N x N
// interior nodes (h = 1/(N+1)). Interior faces carry the harmonic mean 2 k_P k_Q/(k_P+k_Q),
// a boundary face the k of its node. The operator is stored as three FP64 arrays already
// scaled by 1/h^2: the east face aE (at p = N-1 it is the boundary face), the north face aN
// (boundary face at q = N-1) and the diagonal (sum of the four faces). West/south couplings
// are the neighbour's aE/aN, so A is exactly symmetric.
#include "internal.cuh"

#include <cmath>

namespace fcgno {

__global__ void assemble_kernel(int N, size_t n, size_t total, const double* __restrict__ k,
                                double* __restrict__ aE, double* __restrict__ aN,
                                double* __restrict__ diag, double* __restrict__ logk, float* __restrict__ logk32,
                                double* __restrict__ kinv) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const size_t b = i / n;
  const int x = (int)(i - b * n);
  assemble_point(N, x, k + b * n, i, aE, aN, diag, logk, logk32, kinv);
}

__global__ void apply_A_kernel(int N, size_t n, size_t total, const double* __restrict__ aE,
                               const double* __restrict__ aN, const double* __restrict__ diag,
                               const double* __restrict__ x, double* __restrict__ y) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const size_t b = i / n;
  const int xi = (int)(i - b * n);
  const int q = xi / N, p = xi - q * N;
  double acc = diag[i] * x[i];
  if (p < N - 1) acc = fma(-aE[i], x[i + 1], acc);
  if (p > 0) acc = fma(-aE[i - 1], x[i - 1], acc);
  if (q < N - 1) acc = fma(-aN[i], x[i + N], acc);
  if (q > 0) acc = fma(-aN[i - N], x[i - N], acc);
  y[i] = acc;
}

__global__ void rms_kernel(const double* __restrict__ r, size_t n, double* __restrict__ rms) {
  __shared__ double scratch[32];
  const double* rb = r + blockIdx.x * n;
  double v[1] = {0.0};
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) v[0] = fma(rb[i], rb[i], v[0]);
  block_sum<double, 1>(v, scratch);
  if (threadIdx.x == 0) rms[blockIdx.x] = sqrt(v[0] / (double)n);
}

// r = b - A u and e = u_star - u for every instance (the training pairs of random residuals).
__global__ void residual_pair_kernel(int N, size_t n, size_t total, const double* __restrict__ aE,
                                     const double* __restrict__ aN, const double* __restrict__ diag,
                                     const double* __restrict__ b, const double* __restrict__ u,
                                     const double* __restrict__ ustar, double* __restrict__ r,
                                     double* __restrict__ e) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const size_t bi = i / n;
  const int xi = (int)(i - bi * n);
  const int q = xi / N, p = xi - q * N;
  double acc = diag[i] * u[i];
  if (p < N - 1) acc = fma(-aE[i], u[i + 1], acc);
  if (p > 0) acc = fma(-aE[i - 1], u[i - 1], acc);
  if (q < N - 1) acc = fma(-aN[i], u[i + N], acc);
  if (q > 0) acc = fma(-aN[i - N], u[i - N], acc);
  r[i] = b[i] - acc;
  e[i] = ustar[i] - u[i];
}

fcgno_status launch_apply_A(const fcgno_op* op, const double* x, double* y, cudaStream_t st) {
  const size_t total = op->n * op->B;
  apply_A_kernel<<<ceil_div(total, 256), 256, 0, st>>>(op->N, op->n, total, op->aE, op->aN, op->diag, x, y);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

fcgno_status launch_assemble(const fcgno_op* op, size_t off, size_t total, const double* k, cudaStream_t st) {
  assemble_kernel<<<ceil_div(total, 256), 256, 0, st>>>(op->N, op->n, total, k, op->aE + off, op->aN + off,
                                                        op->diag + off, op->logk + off, op->logk32 + off,
                                                        op->kinv + off);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

fcgno_status launch_rms(const double* r, int B, size_t n, double* rms, cudaStream_t st) {
  rms_kernel<<<B, 512, 0, st>>>(r, n, rms);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

}  // namespace fcgno

using namespace fcgno;

// An assembled operator holds aE, aN, the diagonal, log k and 1/k in FP64 and log k in FP32.
size_t fcgno::operator_bytes(size_t n, int B) { return 5 * n * B * sizeof(double) + n * B * sizeof(float); }

extern "C" fcgno_status fcgno_assemble(int N, int batch, const double* k, void* stream, fcgno_op_t* out) {
  if (N < 2 || batch < 1 || !k || !out) {
    set_last_error("fcgno_assemble: need N >= 2, batch >= 1, non-null k and out");
    return FCGNO_EINVAL;
  }
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  fcgno_op* op = new fcgno_op();
  op->N = N;
  op->B = batch;
  op->n = (size_t)N * N;
  const size_t bytes = op->n * batch * sizeof(double);
  if (cudaMalloc(&op->aE, bytes) != cudaSuccess || cudaMalloc(&op->aN, bytes) != cudaSuccess ||
      cudaMalloc(&op->diag, bytes) != cudaSuccess || cudaMalloc(&op->logk, bytes) != cudaSuccess ||
      cudaMalloc(&op->logk32, bytes / 2) != cudaSuccess || cudaMalloc(&op->kinv, bytes) != cudaSuccess) {
    cudaGetLastError();
    fcgno_op_destroy(op);
    set_last_error("fcgno_assemble: out of device memory");
    return FCGNO_ENOMEM;
  }
  const fcgno_status rc = launch_assemble(op, 0, op->n * batch, k, st);
  if (rc != FCGNO_OK) {
    fcgno_op_destroy(op);
    return rc;
  }
  *out = op;
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_reassemble(fcgno_op_t op, const double* k, void* stream) {
  if (!op || !k) {
    set_last_error("fcgno_reassemble: null operator or k");
    return FCGNO_EINVAL;
  }
  return launch_assemble(op, 0, op->n * op->B, k, (cudaStream_t)stream);
}

extern "C" fcgno_status fcgno_residual_pair(fcgno_op_t op, const double* b, const double* u, const double* u_star,
                                            double* r_out, double* e_out, void* stream) {
  if (!op || !b || !u || !u_star || !r_out || !e_out || r_out == u || e_out == u) {
    set_last_error("fcgno_residual_pair: null or aliasing arguments");
    return FCGNO_EINVAL;
  }
  const size_t total = op->n * op->B;
  residual_pair_kernel<<<ceil_div(total, 256), 256, 0, (cudaStream_t)stream>>>(
      op->N, op->n, total, op->aE, op->aN, op->diag, b, u, u_star, r_out, e_out);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_apply_A(fcgno_op_t op, const double* x, double* y, void* stream) {
  if (!op || !x || !y || x == y) {
    set_last_error("fcgno_apply_A: null or aliasing arguments");
    return FCGNO_EINVAL;
  }
  return launch_apply_A(op, x, y, (cudaStream_t)stream);
}
