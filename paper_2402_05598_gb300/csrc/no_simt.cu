// Fourier neural operator preconditioner on CUDA cores, FP64 or FP32 (Section 2.4.2,
// Appendix A), plus its hand-written backward for the energy-norm loss of Eq. (11).
//
// Forward, per instance (activations channels-last [B][q][p][C]):
//   v0 = lift_w [r/rms, log k] + lift_b
//   layer l: c = A v (truncated analysis), c' = R_l c (per-mode complex C x C),
//            h = W_l v + b_l + S c' (truncated synthesis), v = GELU(h) (no GELU on the last)
//   z = h^2 rms(r) * (proj2_w . GELU(proj1_w v + proj1_b) + proj2_b)
// The truncated transforms are separable: analysis first sums over q (x2-frequencies
// k2 = 0..M-1), then over p (x1-frequencies j -> k1 = j or j-2M); synthesis runs the two
// stages in reverse. Twiddles come from tables built on the device with sincospi of the
// exactly reduced phase (k x mod N) / N.
#include "internal.cuh"

#include <vector>
#include <cmath>

namespace fcgno {

template <typename T>
struct Cx {
  T re, im;
};

// ------------------------------------ workspace ----------------------------------------
struct SimtBuffers {
  size_t cap_elems = 0;  // B * n * C capacity of one activation
  size_t cap_spec = 0;   // B * Kx * Ky * C complex capacity
  size_t cap_mid = 0;    // B * Ky * N * C complex capacity
  void* va = nullptr;    // activations (T)
  void* vb = nullptr;
  void* mid = nullptr;   // Z or U (complex T)
  void* spec = nullptr;  // analysis output (complex T)
  void* spec2 = nullptr; // mixed (complex T)
};

struct TwiddleTable {
  int N = 0, M = 0;
  double* tw1 = nullptr;  // [N][Kx][2]  (cos, sin) of 2 pi k1(j) p / N
  double* tw2 = nullptr;  // [N][Ky][2]  (cos, sin) of 2 pi k2 q / N
  float* tw1f = nullptr;
  float* tw2f = nullptr;
};

struct TrainBuffers {
  size_t cap_pts = 0;  // B * n
  int L = 0, C = 0, Cp = 0, Kx = 0, Ky = 0, B = 0;
  void* x0 = nullptr;                 // [pts][2]  (r/rms, log k)
  std::vector<void*> vin;             // L+1 activations [pts][C] (inputs of each layer, vin[L] = last output)
  std::vector<void*> hpre;            // L pre-activations [pts][C] (one scratch buffer when recomputing)
  bool recompute = false;             // pre-activations rebuilt in the backward instead of kept
  bool no_hpre = false;               // BF16 step: its pre-activations are kept in 16 bits elsewhere
  std::vector<void*> chat;            // L analysis outputs [B][Kx][Ky][C] complex
  void* apre = nullptr;               // [pts][Cp] decoder pre-activation
  void* ghid = nullptr;               // [pts][Cp] GELU(apre)
  void* gz = nullptr;                 // [pts] dL/dzt
  void* g0 = nullptr;                 // [pts][C] gradient buffers
  void* g1 = nullptr;
  void* gtmp = nullptr;               // [pts][C]
  void* partials = nullptr;           // [G][...] reduction partials
  size_t partial_cap = 0;
  double* dvec = nullptr;             // FP64 [pts] x3: d = z - e, A d, A e
  double* zbuf = nullptr;             // FP64 [pts]
  double* rms = nullptr;              // [B]
  double* lossb = nullptr;            // [B][2] energy norms
};

}  // namespace fcgno

struct fcgno::NoWorkspace {
  SimtBuffers f64, f32;
  TwiddleTable tw;
  TrainBuffers tr;
};

namespace fcgno {

static void cfree(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void no_workspace_free(fcgno_model* m) {
  if (!m->ws) return;
  NoWorkspace* w = m->ws;
  for (SimtBuffers* s : {&w->f64, &w->f32}) {
    cfree(s->va);
    cfree(s->vb);
    cfree(s->mid);
    cfree(s->spec);
    cfree(s->spec2);
  }
  void* t[] = {w->tw.tw1, w->tw.tw2, w->tw.tw1f, w->tw.tw2f};
  for (void* p : t)
    if (p) cudaFree(p);
  TrainBuffers& tr = w->tr;
  cfree(tr.x0);
  for (auto& p : tr.vin) cfree(p);
  for (auto& p : tr.hpre) cfree(p);
  for (auto& p : tr.chat) cfree(p);
  void** more[] = {&tr.apre, &tr.ghid, &tr.gz, &tr.g0, &tr.g1, &tr.gtmp, &tr.partials,
                   (void**)&tr.dvec, (void**)&tr.zbuf, (void**)&tr.rms, (void**)&tr.lossb};
  for (void** p : more) cfree(*p);
  delete w;
  m->ws = nullptr;
}

__global__ void twiddle_kernel(int N, int M, double* tw1, double* tw2, float* tw1f, float* tw2f) {
  const int Kx = 2 * M, Ky = M;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < N * Kx) {
    const int x = idx / Kx, j = idx % Kx;
    const long long k1 = (j < M) ? j : j - 2 * M;
    const long long ph = ((k1 % N + N) % N) * x % N;
    double s, c;
    sincospi(2.0 * (double)ph / (double)N, &s, &c);
    tw1[2 * idx] = c;
    tw1[2 * idx + 1] = s;
    tw1f[2 * idx] = (float)c;
    tw1f[2 * idx + 1] = (float)s;
  }
  if (idx < N * Ky) {
    const int x = idx / Ky, k2 = idx % Ky;
    const long long ph = (long long)k2 * x % N;
    double s, c;
    sincospi(2.0 * (double)ph / (double)N, &s, &c);
    tw2[2 * idx] = c;
    tw2[2 * idx + 1] = s;
    tw2f[2 * idx] = (float)c;
    tw2f[2 * idx + 1] = (float)s;
  }
}

static fcgno_status ensure_twiddles(fcgno_model* m, int N, cudaStream_t st) {
  if (!m->ws) m->ws = new NoWorkspace();
  TwiddleTable& t = m->ws->tw;
  const int M = m->desc.modes;
  if (t.N == N && t.M == M) return FCGNO_OK;
  if (t.tw1) cudaFree(t.tw1);
  if (t.tw2) cudaFree(t.tw2);
  if (t.tw1f) cudaFree(t.tw1f);
  if (t.tw2f) cudaFree(t.tw2f);
  t = TwiddleTable();
  const size_t n1 = (size_t)N * 2 * M * 2, n2 = (size_t)N * M * 2;
  if (cudaMalloc(&t.tw1, n1 * 8) != cudaSuccess || cudaMalloc(&t.tw2, n2 * 8) != cudaSuccess ||
      cudaMalloc(&t.tw1f, n1 * 4) != cudaSuccess || cudaMalloc(&t.tw2f, n2 * 4) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("twiddle tables: out of device memory");
    return FCGNO_ENOMEM;
  }
  twiddle_kernel<<<ceil_div((size_t)N * 2 * M, 256), 256, 0, st>>>(N, M, t.tw1, t.tw2, t.tw1f, t.tw2f);
  FCGNO_LAUNCHED();
  t.N = N;
  t.M = M;
  m->gen++;
  return FCGNO_OK;
}

template <typename T>
static void tw_ptrs(const TwiddleTable& t, const T*& tw1, const T*& tw2);
template <>
void tw_ptrs<double>(const TwiddleTable& t, const double*& tw1, const double*& tw2) {
  tw1 = t.tw1;
  tw2 = t.tw2;
}
template <>
void tw_ptrs<float>(const TwiddleTable& t, const float*& tw1, const float*& tw2) {
  tw1 = t.tw1f;
  tw2 = t.tw2f;
}

template <typename T>
__device__ __forceinline__ T act_gelu(T x);
template <>
__device__ __forceinline__ double act_gelu<double>(double x) { return gelu_d(x); }
template <>
__device__ __forceinline__ float act_gelu<float>(float x) { return gelu_f(x); }
template <typename T>
__device__ __forceinline__ T act_gelu_grad(T x);
template <>
__device__ __forceinline__ double act_gelu_grad<double>(double x) { return gelu_grad_d(x); }
template <>
__device__ __forceinline__ float act_gelu_grad<float>(float x) { return gelu_grad_f(x); }

__device__ __forceinline__ bool inactive(const int* active, int b) { return active && active[b] >= 0; }

// ------------------------------------ forward kernels ----------------------------------
// v0[b][x][c] = lw[c][0] r[x]/rms + lw[c][1] log k[x] + lb[c]; optionally stores (r/rms, log k).
template <typename T>
__global__ void lift_kernel(int B, size_t n, int C, const double* __restrict__ r, const double* __restrict__ logk,
                            const double* __restrict__ rms, const int* __restrict__ active,
                            const T* __restrict__ lw, const T* __restrict__ lb, T* __restrict__ v,
                            T* __restrict__ x0save) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;  // point index over B*n
  const int b = blockIdx.y;
  if (i >= n || inactive(active, b)) return;
  const double s = rms[b];
  const T rh = (s > 0.0) ? (T)(r[(size_t)b * n + i] / s) : (T)0;
  const T lk = (T)logk[(size_t)b * n + i];
  T* out = v + ((size_t)b * n + i) * C;
  for (int c = 0; c < C; ++c) out[c] = lw[2 * c] * rh + lw[2 * c + 1] * lk + lb[c];
  if (x0save) {
    x0save[((size_t)b * n + i) * 2] = rh;
    x0save[((size_t)b * n + i) * 2 + 1] = lk;
  }
}

// Z[b][k2][p][c] = sum_q v[b][q][p][c] exp(-2 pi i k2 q / N)   (thread per (p, c))
template <typename T, int KY>
__global__ void analysis_q_kernel(int N, int C, const int* __restrict__ active, const T* __restrict__ v,
                                  const T* __restrict__ tw2, Cx<T>* __restrict__ Z) {
  const int b = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;  // p*C + c
  if (j >= N * C || inactive(active, b)) return;
  const size_t n = (size_t)N * N;
  T re[KY], im[KY];
#pragma unroll
  for (int k = 0; k < KY; ++k) re[k] = im[k] = (T)0;
  const T* vb = v + (size_t)b * n * C + j;
  for (int q = 0; q < N; ++q) {
    const T x = vb[(size_t)q * N * C];
    const T* t = tw2 + (size_t)q * KY * 2;
#pragma unroll
    for (int k = 0; k < KY; ++k) {
      re[k] += x * t[2 * k];
      im[k] -= x * t[2 * k + 1];
    }
  }
  Cx<T>* zb = Z + (size_t)b * KY * N * C + j;
#pragma unroll
  for (int k = 0; k < KY; ++k) zb[(size_t)k * N * C] = Cx<T>{re[k], im[k]};
}

// c[b][j][k2][c] = scale(k2) * sum_p Z[b][k2][p][c] exp(-2 pi i k1(j) p / N)
// scale(k2) = s0 for k2 = 0 and s1 otherwise.   (block per (k2, b), thread per (j, c))
template <typename T>
__global__ void analysis_p_kernel(int N, int C, int Kx, int Ky, T s0, T s1, const int* __restrict__ active,
                                  const Cx<T>* __restrict__ Z, const T* __restrict__ tw1, Cx<T>* __restrict__ out) {
  const int k2 = blockIdx.x, b = blockIdx.y;
  if (inactive(active, b)) return;
  const T sc = (k2 == 0) ? s0 : s1;
  const Cx<T>* zb = Z + ((size_t)b * Ky + k2) * N * C;
  for (int t = threadIdx.x; t < Kx * C; t += blockDim.x) {
    const int j = t / C, c = t % C;
    T re = 0, im = 0;
    for (int p = 0; p < N; ++p) {
      const Cx<T> z = zb[(size_t)p * C + c];
      const T cs = tw1[((size_t)p * Kx + j) * 2], sn = tw1[((size_t)p * Kx + j) * 2 + 1];
      re += z.re * cs + z.im * sn;
      im += z.im * cs - z.re * sn;
    }
    out[(((size_t)b * Kx + j) * Ky + k2) * C + c] = Cx<T>{re * sc, im * sc};
  }
}

// Per-mode complex channel mixing. conj_t = false: out[o] = sum_i in[i] R[i][o];
// conj_t = true (adjoint): out[i] = sum_o conj(R[i][o]) in[o].  R = [mode][i][o][2].
template <typename T>
__global__ void mix_kernel(int B, int C, int nmodes, const int* __restrict__ active, const Cx<T>* __restrict__ in,
                           const T* __restrict__ R, Cx<T>* __restrict__ out, int conj_t) {
  extern __shared__ unsigned char smraw[];
  Cx<T>* Rs = reinterpret_cast<Cx<T>*>(smraw);  // C*C
  const int mode = blockIdx.x;
  const T* Rm = R + (size_t)mode * C * C * 2;
  for (int t = threadIdx.x; t < C * C; t += blockDim.x) Rs[t] = Cx<T>{Rm[2 * t], Rm[2 * t + 1]};
  __syncthreads();
  for (int t = threadIdx.x; t < B * C; t += blockDim.x) {
    const int b = t / C, o = t % C;
    if (inactive(active, b)) continue;
    const Cx<T>* x = in + ((size_t)b * nmodes + mode) * C;
    T re = 0, im = 0;
    if (!conj_t) {
      for (int i = 0; i < C; ++i) {
        const Cx<T> a = x[i], w = Rs[i * C + o];
        re += a.re * w.re - a.im * w.im;
        im += a.re * w.im + a.im * w.re;
      }
    } else {
      for (int i = 0; i < C; ++i) {  // here o plays the role of the input index of R
        const Cx<T> a = x[i], w = Rs[o * C + i];
        re += a.re * w.re + a.im * w.im;
        im += a.im * w.re - a.re * w.im;
      }
    }
    out[((size_t)b * nmodes + mode) * C + o] = Cx<T>{re, im};
  }
}

// U[b][k2][p][c] = sum_j c'[b][j][k2][c] exp(+2 pi i k1(j) p / N)   (thread per (p, c))
template <typename T>
__global__ void synthesis_p_kernel(int N, int C, int Kx, int Ky, const int* __restrict__ active,
                                   const Cx<T>* __restrict__ cin, const T* __restrict__ tw1, Cx<T>* __restrict__ U) {
  const int jpc = blockIdx.x * blockDim.x + threadIdx.x;
  const int k2 = blockIdx.y, b = blockIdx.z;
  if (jpc >= N * C || inactive(active, b)) return;
  const int p = jpc / C, c = jpc % C;
  T re = 0, im = 0;
  for (int j = 0; j < Kx; ++j) {
    const Cx<T> a = cin[(((size_t)b * Kx + j) * Ky + k2) * C + c];
    const T cs = tw1[((size_t)p * Kx + j) * 2], sn = tw1[((size_t)p * Kx + j) * 2 + 1];
    re += a.re * cs - a.im * sn;
    im += a.re * sn + a.im * cs;
  }
  U[(((size_t)b * Ky + k2) * N + p) * C + c] = Cx<T>{re, im};
}

// out[b][x][o] = act( sum_i Wt(o,i) v[b][x][i] + bias[o] + sum_k2 w(k2) Re(U[b][k2][p][o] e^{+2 pi i k2 q/N}) )
// Wt(o,i) = W[o][i] (transposed = 0) or W[i][o] (transposed = 1); w(0) = w0, w(k2>0) = w1.
// hsave (optional) receives the pre-activation. Block: 256 threads = (256/C) points x C.
template <typename T>
__global__ void synthesis_q_pointwise_kernel(int N, int C, int Ky, const int* __restrict__ active,
                                             const T* __restrict__ v, const Cx<T>* __restrict__ U,
                                             const T* __restrict__ tw2, const T* __restrict__ W,
                                             int transposed, const T* __restrict__ bias, T w0, T w1,
                                             int activate, T* __restrict__ out, T* __restrict__ hsave) {
  extern __shared__ unsigned char smraw[];
  T* Ws = reinterpret_cast<T*>(smraw);  // C*C, stored as Ws[o*C+i]
  T* vs = Ws + C * C;                   // (points per block) * C
  const int b = blockIdx.y;
  if (inactive(active, b)) return;
  const size_t n = (size_t)N * N;
  const int ppb = blockDim.x / C;
  for (int t = threadIdx.x; t < C * C; t += blockDim.x) {
    const int o = t / C, i = t % C;
    Ws[t] = transposed ? W[i * C + o] : W[o * C + i];
  }
  const size_t x0 = (size_t)blockIdx.x * ppb;
  for (int t = threadIdx.x; t < ppb * C; t += blockDim.x) {
    const size_t x = x0 + t / C;
    vs[t] = (x < n) ? v[((size_t)b * n + x) * C + (t % C)] : (T)0;
  }
  __syncthreads();
  const int lp = threadIdx.x / C, o = threadIdx.x % C;
  const size_t x = x0 + lp;
  if (lp >= ppb || x >= n) return;
  const int q = (int)(x / N), p = (int)(x % N);
  T acc = bias ? bias[o] : (T)0;
  for (int i = 0; i < C; ++i) acc += Ws[o * C + i] * vs[lp * C + i];
  const Cx<T>* Ub = U + (size_t)b * Ky * N * C;  // U is [B][Ky][N][C]
  for (int k2 = 0; k2 < Ky; ++k2) {
    const Cx<T> u = Ub[((size_t)k2 * N + p) * C + o];
    const T cs = tw2[((size_t)q * Ky + k2) * 2], sn = tw2[((size_t)q * Ky + k2) * 2 + 1];
    acc += (k2 == 0 ? w0 : w1) * (u.re * cs - u.im * sn);
  }
  const size_t oi = ((size_t)b * n + x) * C + o;
  if (hsave) hsave[oi] = acc;
  out[oi] = activate ? act_gelu<T>(acc) : acc;
}

// z[b][x] = h^2 rms * (p2 . GELU(P1 v + p1) + p2b) (hh = h^2), times 1/k[b][x] when kinv is
// given (output_scale 1); optional saves of the decoder's pre-activation and GELU output.
template <typename T>
__global__ void project_kernel(size_t n, int C, int Cp, const int* __restrict__ active, const T* __restrict__ v,
                               const T* __restrict__ P1, const T* __restrict__ p1, const T* __restrict__ p2,
                               const T* __restrict__ p2b, const double* __restrict__ rms, double hh,
                               const double* __restrict__ kinv, double* __restrict__ z, T* __restrict__ asave,
                               T* __restrict__ gsave, double* __restrict__ ztsave) {
  extern __shared__ unsigned char smraw[];
  T* P1s = reinterpret_cast<T*>(smraw);  // Cp*C
  for (int t = threadIdx.x; t < Cp * C; t += blockDim.x) P1s[t] = P1[t];
  __syncthreads();
  const int b = blockIdx.y;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= n || inactive(active, b)) return;
  const T* vx = v + ((size_t)b * n + x) * C;
  T vr[64];
  for (int c = 0; c < C; ++c) vr[c] = vx[c];
  T zt = p2b[0];
  for (int h = 0; h < Cp; ++h) {
    T a = p1[h];
    for (int c = 0; c < C; ++c) a += P1s[h * C + c] * vr[c];
    const T g = act_gelu<T>(a);
    if (asave) {
      asave[((size_t)b * n + x) * Cp + h] = a;
      gsave[((size_t)b * n + x) * Cp + h] = g;
    }
    zt += p2[h] * g;
  }
  if (ztsave) ztsave[(size_t)b * n + x] = (double)zt;
  const double sc = rms[b] * hh;
  z[(size_t)b * n + x] = (kinv ? sc * kinv[(size_t)b * n + x] : sc) * (double)zt;
}

// ------------------------------------ host: forward ------------------------------------
template <typename T>
struct Wp {  // pointers into a blob of T
  const T *lift_w, *lift_b, *proj1_w, *proj1_b, *proj2_w, *proj2_b;
  const T *w[16], *b[16], *r[16];
};
template <typename T>
static Wp<T> wptrs(const fcgno_model* m, const T* base) {
  BlobLayout L = blob_layout(m->desc);
  Wp<T> p;
  p.lift_w = base + L.lift_w;
  p.lift_b = base + L.lift_b;
  p.proj1_w = base + L.proj1_w;
  p.proj1_b = base + L.proj1_b;
  p.proj2_w = base + L.proj2_w;
  p.proj2_b = base + L.proj2_b;
  for (int l = 0; l < m->desc.layers; ++l) {
    p.w[l] = base + L.w[l];
    p.b[l] = base + L.b[l];
    p.r[l] = base + L.r[l];
  }
  return p;
}

// Elements of the CUDA-core preconditioner's buffers for a batch of B on an N x N grid:
// two activation ping-pong buffers (B n C), the separable-transform intermediate (complex
// B M N C) and two spectral-coefficient buffers (complex B 2M^2 C).
static void simt_elems(int N, int B, const fcgno_model_desc& d, size_t& elems, size_t& mid, size_t& spec) {
  const size_t C = d.width, M = d.modes;
  elems = (size_t)B * N * N * C;
  spec = (size_t)B * 2 * M * M * C;
  mid = (size_t)B * M * N * C;
}

size_t simt_buffers_bytes(int N, int B, const fcgno_model_desc& d, bool fp64) {
  size_t elems, mid, spec;
  simt_elems(N, B, d, elems, mid, spec);
  return (2 * elems + 2 * mid + 4 * spec) * (fp64 ? 8 : 4);
}

template <typename T>
static fcgno_status ensure_simt(fcgno_model* m, const fcgno_op* op, SimtBuffers& s) {
  size_t elems, mid, spec;
  simt_elems(op->N, op->B, m->desc, elems, mid, spec);
  if (s.cap_elems >= elems && s.cap_spec >= spec && s.cap_mid >= mid) return FCGNO_OK;
  cfree(s.va);
  cfree(s.vb);
  cfree(s.mid);
  cfree(s.spec);
  cfree(s.spec2);
  s.cap_elems = s.cap_spec = s.cap_mid = 0;
  if (cudaMalloc(&s.va, elems * sizeof(T)) != cudaSuccess || cudaMalloc(&s.vb, elems * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&s.mid, mid * 2 * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&s.spec, spec * 2 * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&s.spec2, spec * 2 * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("preconditioner workspace: out of device memory");
    return FCGNO_ENOMEM;
  }
  s.cap_elems = elems;
  s.cap_spec = spec;
  s.cap_mid = mid;
  m->gen++;
  return FCGNO_OK;
}

template <typename T>
static fcgno_status launch_analysis(int N, int B, int C, int M, const int* active, const T* v, Cx<T>* mid,
                                    Cx<T>* out, T s0, T s1, const T* tw1, const T* tw2, cudaStream_t st) {
  const dim3 g1(ceil_div((size_t)N * C, 128), B);
  switch (M) {
#define FCGNO_AQ(KY) \
  case KY: analysis_q_kernel<T, KY><<<g1, 128, 0, st>>>(N, C, active, v, tw2, mid); break;
    FCGNO_AQ(1) FCGNO_AQ(2) FCGNO_AQ(3) FCGNO_AQ(4) FCGNO_AQ(5) FCGNO_AQ(6) FCGNO_AQ(7) FCGNO_AQ(8)
    FCGNO_AQ(9) FCGNO_AQ(10) FCGNO_AQ(11) FCGNO_AQ(12) FCGNO_AQ(13) FCGNO_AQ(14) FCGNO_AQ(15) FCGNO_AQ(16)
#undef FCGNO_AQ
    default:
      set_last_error("modes must be 1..16");
      return FCGNO_EINVAL;
  }
  FCGNO_LAUNCHED();
  const int Kx = 2 * M;
  analysis_p_kernel<T><<<dim3(M, B), std::min(1024, ((Kx * C + 31) / 32) * 32), 0, st>>>(N, C, Kx, M, s0, s1, active,
                                                                                        mid, tw1, out);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

template <typename T>
static fcgno_status launch_synthesis_p(int N, int B, int C, int M, const int* active, const Cx<T>* cin,
                                       const T* tw1, Cx<T>* U, cudaStream_t st) {
  synthesis_p_kernel<T><<<dim3(ceil_div((size_t)N * C, 128), M, B), 128, 0, st>>>(N, C, 2 * M, M, active, cin, tw1, U);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

template <typename T>
static fcgno_status launch_syn_q_pw(int N, int B, int C, int M, const int* active, const T* v, const Cx<T>* U,
                                    const T* tw2, const T* W, int transposed, const T* bias, T w0, T w1, int act,
                                    T* out, T* hsave, cudaStream_t st) {
  const int ppb = 256 / C;
  const size_t smem = (size_t)(C * C + ppb * C) * sizeof(T);
  synthesis_q_pointwise_kernel<T><<<dim3(ceil_div((size_t)N * N, ppb), B), ppb * C, smem, st>>>(
      N, C, M, active, v, U, tw2, W, transposed, bias, w0, w1, act, out, hsave);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

// Runs the forward pass. When `tr` is non-null every intermediate the backward needs is
// saved into it (training); otherwise activations ping-pong in `s`.
template <typename T>
static fcgno_status forward_simt(fcgno_model* m, const fcgno_op* op, const T* wbase, const double* r,
                                 const double* rms, const int* active, double* z, SimtBuffers& s, TrainBuffers* tr,
                                 double* ztsave, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  const int N = op->N, B = op->B, C = d.width, M = d.modes, Cp = d.proj_width, L = d.layers;
  const size_t n = op->n;
  FCGNO_TRY(ensure_twiddles(m, N, st));
  const T *tw1, *tw2;
  tw_ptrs<T>(m->ws->tw, tw1, tw2);
  Wp<T> W = wptrs<T>(m, wbase);
  T* cur = tr ? (T*)tr->vin[0] : (T*)s.va;
  lift_kernel<T><<<dim3(ceil_div(n, 256), B), 256, 0, st>>>(B, n, C, r, op->logk, rms, active, W.lift_w, W.lift_b,
                                                            cur, tr ? (T*)tr->x0 : nullptr);
  FCGNO_LAUNCHED();
  const T inv_n = (T)(1.0 / (double)n);
  for (int l = 0; l < L; ++l) {
    T* nxt = tr ? (T*)tr->vin[l + 1] : ((cur == (T*)s.va) ? (T*)s.vb : (T*)s.va);
    Cx<T>* chat = tr ? (Cx<T>*)tr->chat[l] : (Cx<T>*)s.spec;
    FCGNO_TRY(launch_analysis<T>(N, B, C, M, active, cur, (Cx<T>*)s.mid, chat, inv_n, inv_n, tw1, tw2, st));
    mix_kernel<T><<<2 * M * M, 256, C * C * sizeof(Cx<T>), st>>>(B, C, 2 * M * M, active, chat, W.r[l],
                                                                (Cx<T>*)s.spec2, 0);
    FCGNO_LAUNCHED();
    FCGNO_TRY(launch_synthesis_p<T>(N, B, C, M, active, (Cx<T>*)s.spec2, tw1, (Cx<T>*)s.mid, st));
    FCGNO_TRY(launch_syn_q_pw<T>(N, B, C, M, active, cur, (Cx<T>*)s.mid, tw2, W.w[l], 0, W.b[l], (T)1, (T)2,
                                 l < L - 1, nxt, (tr && !tr->recompute) ? (T*)tr->hpre[l] : nullptr, st));
    cur = nxt;
  }
  const size_t smem = (size_t)Cp * C * sizeof(T);
  project_kernel<T><<<dim3(ceil_div(n, 128), B), 128, smem, st>>>(n, C, Cp, active, cur, W.proj1_w, W.proj1_b,
                                                                   W.proj2_w, W.proj2_b, rms,
                                                                   1.0 / ((double)(N + 1) * (N + 1)),
                                                                   d.output_scale ? op->kinv : nullptr, z,
                                                                   tr ? (T*)tr->apre : nullptr,
                                                                   tr ? (T*)tr->ghid : nullptr, ztsave);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

fcgno_status no_apply_simt(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms,
                           const int* active, double* z, bool fp64, cudaStream_t st) {
  if (m->desc.width > 64 || m->desc.proj_width > 64 || 256 % m->desc.width != 0) {
    set_last_error("CUDA-core preconditioner supports width dividing 256 and <= 64");
    return FCGNO_EINVAL;
  }
  if (!m->ws) m->ws = new NoWorkspace();
  if (fp64) {
    FCGNO_TRY(ensure_simt<double>(m, op, m->ws->f64));
    return forward_simt<double>(m, op, m->w64, r, rms, active, z, m->ws->f64, nullptr, nullptr, st);
  }
  FCGNO_TRY(ensure_simt<float>(m, op, m->ws->f32));
  return forward_simt<float>(m, op, m->w32, r, rms, active, z, m->ws->f32, nullptr, nullptr, st);
}

// ------------------------------------ backward kernels ---------------------------------
// Weight-gradient reduction: partial[g][o][i] = sum_{x in chunk g} A[x][o] V[x][i] and
// partial[g][o][Ci] = sum_x A[x][o]. Points are split into G contiguous chunks (fixed).
template <typename T>
__global__ void outer_reduce_kernel(size_t npts, int Co, int Ci, const T* __restrict__ A, const T* __restrict__ V,
                                    T* __restrict__ partial) {
  extern __shared__ unsigned char smraw[];
  constexpr int kRows = 32;
  T* As = reinterpret_cast<T*>(smraw);  // kRows * Co
  T* Vs = As + kRows * Co;              // kRows * Ci
  const int G = gridDim.x, g = blockIdx.x;
  const size_t chunk = (npts + G - 1) / G;
  const size_t x0 = (size_t)g * chunk, x1 = (x0 + chunk < npts) ? x0 + chunk : npts;
  const int nout = Co * (Ci + 1);
  T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // up to 8 outputs per thread (blockDim * 8 >= nout)
  for (size_t xb = x0; xb < x1; xb += kRows) {
    const int rows = (int)((x1 - xb < (size_t)kRows) ? (x1 - xb) : kRows);
    __syncthreads();
    for (int t = threadIdx.x; t < rows * Co; t += blockDim.x) As[t] = A[(xb + t / Co) * Co + t % Co];
    for (int t = threadIdx.x; t < rows * Ci; t += blockDim.x) Vs[t] = V[(xb + t / Ci) * Ci + t % Ci];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = threadIdx.x + u * blockDim.x;
      if (idx < nout) {
        const int o = idx / (Ci + 1), i = idx % (Ci + 1);
        T s = acc[u];
        if (i < Ci) {
          for (int rr = 0; rr < rows; ++rr) s += As[rr * Co + o] * Vs[rr * Ci + i];
        } else {
          for (int rr = 0; rr < rows; ++rr) s += As[rr * Co + o];
        }
        acc[u] = s;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int idx = threadIdx.x + u * blockDim.x;
    if (idx < nout) partial[(size_t)g * nout + idx] = acc[u];
  }
}

// grad_w[o*Ci+i] = sum_g partial[g][o][i]; grad_b[o] = sum_g partial[g][o][Ci] (grad_b may be null).
// Gr: the gradient's storage type (float, or double for the FP64-output step).
template <typename T, typename Gr>
__global__ void reduce_partials_kernel(int G, int Co, int Ci, const T* __restrict__ partial, Gr* __restrict__ gw,
                                       Gr* __restrict__ gb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nout = Co * (Ci + 1);
  if (idx >= nout) return;
  T s = 0;
  for (int g = 0; g < G; ++g) s += partial[(size_t)g * nout + idx];
  const int o = idx / (Ci + 1), i = idx % (Ci + 1);
  if (i < Ci)
    gw[o * Ci + i] = (Gr)s;
  else if (gb)
    gb[o] = (Gr)s;
}

// Loss pieces: per instance sqrt(d, Ad) and sqrt(e, Ae) with d = z - e; Ad = A d and Ae = A e
// for the energy norm, Ad = d and Ae = e for the 2-norm.
__global__ void loss_dots_kernel(size_t n, const double* __restrict__ d, const double* __restrict__ Ad,
                                 const double* __restrict__ e, const double* __restrict__ Ae, double* __restrict__ out) {
  __shared__ double scratch[64];
  const int b = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const size_t gi = (size_t)b * n + i;
    v[0] = fma(d[gi], Ad[gi], v[0]);
    v[1] = fma(e[gi], Ae[gi], v[1]);
  }
  block_sum<double, 2>(v, scratch);
  if (threadIdx.x == 0) {
    out[2 * b] = sqrt(v[0]);
    out[2 * b + 1] = sqrt(v[1]);
  }
}

__global__ void diff_kernel(size_t total, const double* __restrict__ z, const double* __restrict__ e,
                            double* __restrict__ d) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < total) d[i] = z[i] - e[i];
}

// loss = mean_b ||d_b|| / ||e_b||  (written to *loss as float, or double)
template <typename Gr>
__global__ void loss_value_kernel(int B, const double* __restrict__ norms, Gr* __restrict__ loss) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += norms[2 * b] / norms[2 * b + 1];
  *loss = (Gr)(s / B);
}

// dL/dzt[b][x] = s_b(x) * (1/B) * (A d)_x / (||d|| ||e||) with s = h^2 rms_b (times 1/k[b][x]
// when kinv is given) the output scale z = s zt; A d -> d for the 2-norm
template <typename T>
__global__ void dzt_kernel(int B, size_t n, double hh, const double* __restrict__ Ad,
                           const double* __restrict__ norms, const double* __restrict__ rms,
                           const double* __restrict__ kinv, T* __restrict__ gzt) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)B * n) return;
  const int b = (int)(i / n);
  const double den = norms[2 * b] * norms[2 * b + 1];
  const double sc = kinv ? hh * rms[b] * kinv[i] : hh * rms[b];
  gzt[i] = (den > 0.0) ? (T)(sc * Ad[i] / (den * B)) : (T)0;
}

// Decoder backward: ga[x][h] = gzt[x] p2[h] GELU'(a[x][h]); gv[x][c] = sum_h ga[x][h] P1[h][c].
template <typename T>
__global__ void project_bwd_kernel(size_t npts, int C, int Cp, const T* __restrict__ gzt, const T* __restrict__ apre,
                                   const T* __restrict__ P1, const T* __restrict__ p2, T* __restrict__ ga,
                                   T* __restrict__ gv) {
  extern __shared__ unsigned char smraw[];
  T* P1s = reinterpret_cast<T*>(smraw);
  for (int t = threadIdx.x; t < Cp * C; t += blockDim.x) P1s[t] = P1[t];
  __syncthreads();
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= npts) return;
  T gah[64];
  const T g = gzt[x];
  for (int h = 0; h < Cp; ++h) {
    gah[h] = g * p2[h] * act_gelu_grad<T>(apre[x * Cp + h]);
    ga[x * Cp + h] = gah[h];
  }
  for (int c = 0; c < C; ++c) {
    T s = 0;
    for (int h = 0; h < Cp; ++h) s += gah[h] * P1s[h * C + c];
    gv[x * C + c] = s;
  }
}

// gh = gv * act'(h) (in place into gh)
template <typename T>
__global__ void act_bwd_kernel(size_t total, const T* __restrict__ gv, const T* __restrict__ h, int activate,
                               T* __restrict__ gh) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  gh[i] = activate ? gv[i] * act_gelu_grad<T>(h[i]) : gv[i];
}

// dR[mode][i][o] = sum_b conj(c[b][mode][i]) g[b][mode][o]   (block per mode, thread per (i,o))
template <typename T, typename Gr>
__global__ void spectral_wgrad_kernel(int B, int C, int nmodes, const Cx<T>* __restrict__ c, const Cx<T>* __restrict__ g,
                                      Gr* __restrict__ dR) {
  const int mode = blockIdx.x;
  for (int t = threadIdx.x; t < C * C; t += blockDim.x) {
    const int i = t / C, o = t % C;
    T re = 0, im = 0;
    for (int b = 0; b < B; ++b) {
      const Cx<T> a = c[((size_t)b * nmodes + mode) * C + i];
      const Cx<T> w = g[((size_t)b * nmodes + mode) * C + o];
      re += a.re * w.re + a.im * w.im;
      im += a.re * w.im - a.im * w.re;
    }
    dR[((size_t)mode * C * C + t) * 2] = (Gr)re;
    dR[((size_t)mode * C * C + t) * 2 + 1] = (Gr)im;
  }
}

__global__ void add_kernel(size_t total, const void* a, void* out, int fp64) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  if (fp64)
    ((double*)out)[i] += ((const double*)a)[i];
  else
    ((float*)out)[i] += ((const float*)a)[i];
}

// ------------------------------------ host: training -----------------------------------
static fcgno_status ensure_train(fcgno_model* m, const fcgno_op* op, size_t esz, bool no_hpre = false) {
  TrainBuffers& t = m->ws->tr;
  const fcgno_model_desc& d = m->desc;
  const size_t pts = (size_t)op->B * op->n;
  const int Kx = 2 * d.modes, Ky = d.modes;
  // Activation checkpointing: the forward keeps every layer's input and its analysis output
  // (small); the L pre-activations (pts x C each) are either kept too or rebuilt one layer at a
  // time in the backward. Automatic mode rebuilds them when keeping them would take more than
  // kKeepBudget bytes.
  constexpr size_t kKeepBudget = (size_t)2 << 30;
  const bool recompute = m->train_recompute == 1 ||
                         (m->train_recompute == 0 && pts * d.width * esz * (size_t)d.layers > kKeepBudget);
  if (t.cap_pts == pts * esz && t.L == d.layers && t.C == d.width && t.Cp == d.proj_width && t.Kx == Kx &&
      t.B == op->B && t.recompute == recompute && t.no_hpre == no_hpre)
    return FCGNO_OK;
  // release and reallocate
  cfree(t.x0);
  for (auto& p : t.vin) cfree(p);
  for (auto& p : t.hpre) cfree(p);
  for (auto& p : t.chat) cfree(p);
  void** more[] = {&t.apre, &t.ghid, &t.gz, &t.g0, &t.g1, &t.gtmp, &t.partials,
                   (void**)&t.dvec, (void**)&t.zbuf, (void**)&t.rms, (void**)&t.lossb};
  for (void** p : more) cfree(*p);
  t.vin.assign(d.layers + 1, nullptr);
  t.hpre.assign(no_hpre ? 0 : (recompute ? 1 : d.layers), nullptr);
  t.chat.assign(d.layers, nullptr);
  bool ok = true;
  auto al = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
  };
  const size_t C = d.width, Cp = d.proj_width;
  al(&t.x0, pts * 2 * esz);
  for (auto& p : t.vin) al(&p, pts * C * esz);
  for (auto& p : t.hpre) al(&p, pts * C * esz);
  for (auto& p : t.chat) al(&p, (size_t)op->B * Kx * Ky * C * 2 * esz);
  al(&t.apre, pts * Cp * esz);
  al(&t.ghid, pts * Cp * esz);
  al(&t.gz, pts * esz);
  al(&t.g0, pts * std::max(C, Cp) * esz);
  al(&t.g1, pts * std::max(C, Cp) * esz);
  al(&t.gtmp, pts * std::max(C, Cp) * esz);
  t.partial_cap = (size_t)1024 * (std::max(C, Cp) * (std::max(C, Cp) + 1));
  al(&t.partials, t.partial_cap * esz);
  al((void**)&t.dvec, pts * 3 * sizeof(double));
  al((void**)&t.zbuf, pts * sizeof(double));
  al((void**)&t.rms, op->B * sizeof(double));
  al((void**)&t.lossb, op->B * 2 * sizeof(double));
  if (!ok) {
    cudaGetLastError();
    set_last_error("training workspace: out of device memory");
    t.cap_pts = 0;
    return FCGNO_ENOMEM;
  }
  t.cap_pts = pts * esz;
  t.recompute = recompute;
  t.no_hpre = no_hpre;
  t.L = d.layers;
  t.C = d.width;
  t.Cp = d.proj_width;
  t.Kx = Kx;
  t.Ky = Ky;
  t.B = op->B;
  return FCGNO_OK;
}

template <typename T, typename Gr>
static fcgno_status outer_reduce(size_t npts, int Co, int Ci, const T* A, const T* V, T* partials, Gr* gw,
                                 Gr* gb, cudaStream_t st) {
  const int G = 512;
  const int threads = 256;
  if (Co * (Ci + 1) > threads * 8) {
    set_last_error("outer_reduce: too many outputs");
    return FCGNO_EINVAL;
  }
  const size_t smem = (size_t)32 * (Co + Ci) * sizeof(T);
  outer_reduce_kernel<T><<<G, threads, smem, st>>>(npts, Co, Ci, A, V, partials);
  FCGNO_LAUNCHED();
  reduce_partials_kernel<T, Gr><<<ceil_div((size_t)Co * (Ci + 1), 256), 256, 0, st>>>(G, Co, Ci, partials, gw, gb);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

// Loss (FP64) of the forward output in t.zbuf and the decoder's backward: the decoder's
// weight gradients, and the gradient of the last Fourier layer's output (FP32 or FP64,
// [B][N][N][C]) left in t.g0. `grad` is zeroed first. vL: the last layer's output.
template <typename T, typename Gr>
static fcgno_status loss_and_decoder_bwd(fcgno_model* m, fcgno_op* op, const double* e, Gr* loss, Gr* grad,
                                         bool l2, const T* vL, const Wp<T>& W, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  const int N = op->N, B = op->B, C = d.width, Cp = d.proj_width;
  const size_t n = op->n, pts = (size_t)B * n;
  TrainBuffers& t = m->ws->tr;
  BlobLayout BL = blob_layout(d);
  // d = z - e, then A d and A e (energy norm, Eq. (11)) or d and e themselves (2-norm of the
  // L2 ablation loss)
  double* dv = t.dvec;
  const double* Ad = dv;
  const double* Ae = e;
  diff_kernel<<<ceil_div(pts, 256), 256, 0, st>>>(pts, t.zbuf, e, dv);
  FCGNO_LAUNCHED();
  if (!l2) {
    FCGNO_TRY(launch_apply_A(op, dv, t.dvec + pts, st));
    FCGNO_TRY(launch_apply_A(op, e, t.dvec + 2 * pts, st));
    Ad = t.dvec + pts;
    Ae = t.dvec + 2 * pts;
  }
  loss_dots_kernel<<<B, 256, 0, st>>>(n, dv, Ad, e, Ae, t.lossb);
  FCGNO_LAUNCHED();
  loss_value_kernel<Gr><<<1, 32, 0, st>>>(B, t.lossb, loss);
  FCGNO_LAUNCHED();
  FCGNO_CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(Gr) * BL.total, st));
  T* gzt = (T*)t.gz;
  dzt_kernel<T><<<ceil_div(pts, 256), 256, 0, st>>>(B, n, 1.0 / ((double)(N + 1) * (N + 1)), Ad, t.lossb, t.rms,
                                                    d.output_scale ? op->kinv : nullptr, gzt);
  FCGNO_LAUNCHED();
  // decoder: proj2 grads (A = gzt [pts][1], V = GELU(a) [pts][Cp])
  FCGNO_TRY(outer_reduce<T>(pts, 1, Cp, gzt, (const T*)t.ghid, (T*)t.partials, grad + BL.proj2_w,
                            grad + BL.proj2_b, st));
  T* ga = (T*)t.gtmp;
  T* gv = (T*)t.g0;
  project_bwd_kernel<T><<<ceil_div(pts, 128), 128, (size_t)Cp * C * sizeof(T), st>>>(pts, C, Cp, gzt, (const T*)t.apre,
                                                                                     W.proj1_w, W.proj2_w, ga, gv);
  FCGNO_LAUNCHED();
  FCGNO_TRY(outer_reduce<T>(pts, Cp, C, ga, vL, (T*)t.partials, grad + BL.proj1_w, grad + BL.proj1_b, st));
  return FCGNO_OK;
}

template <typename T, typename Gr>
static fcgno_status train_impl(fcgno_model* m, fcgno_op* op, const double* r, const double* e, Gr* loss,
                               Gr* grad, bool l2, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  const int N = op->N, B = op->B, C = d.width, M = d.modes, L = d.layers;
  const size_t n = op->n, pts = (size_t)B * n;
  const int Kx = 2 * M, Ky = M, nmodes = Kx * Ky;
  FCGNO_TRY(ensure_train(m, op, sizeof(T)));
  SimtBuffers& s = (sizeof(T) == 8) ? m->ws->f64 : m->ws->f32;
  FCGNO_TRY(ensure_simt<T>(m, op, s));
  TrainBuffers& t = m->ws->tr;
  const T* wbase = (sizeof(T) == 8) ? (const T*)m->w64 : (const T*)m->w32;
  Wp<T> W = wptrs<T>(m, wbase);
  BlobLayout BL = blob_layout(d);
  // forward with saves
  FCGNO_TRY(launch_rms(r, B, n, t.rms, st));
  FCGNO_TRY(forward_simt<T>(m, op, wbase, r, t.rms, nullptr, t.zbuf, s, &t, nullptr, st));
  FCGNO_TRY((loss_and_decoder_bwd<T, Gr>(m, op, e, loss, grad, l2, (const T*)t.vin[L], W, st)));
  // backward
  const T *tw1, *tw2;
  tw_ptrs<T>(m->ws->tw, tw1, tw2);
  T* gv = (T*)t.g0;
  const T inv_n = (T)(1.0 / (double)n);
  T* gh = (T*)t.g1;
  for (int l = L - 1; l >= 0; --l) {
    const T* hpre = (const T*)t.hpre[t.recompute ? 0 : l];
    if (t.recompute) {
      // rebuild layer l's pre-activation from its kept input and analysis output: the same
      // kernels on the same inputs as the forward, so the values are bit-identical (the
      // layer output, rewritten into vin[l + 1], is unchanged)
      mix_kernel<T><<<nmodes, 256, C * C * sizeof(Cx<T>), st>>>(B, C, nmodes, nullptr, (const Cx<T>*)t.chat[l],
                                                                 W.r[l], (Cx<T>*)s.spec2, 0);
      FCGNO_LAUNCHED();
      FCGNO_TRY(launch_synthesis_p<T>(N, B, C, M, nullptr, (Cx<T>*)s.spec2, tw1, (Cx<T>*)s.mid, st));
      FCGNO_TRY(launch_syn_q_pw<T>(N, B, C, M, nullptr, (const T*)t.vin[l], (Cx<T>*)s.mid, tw2, W.w[l], 0, W.b[l],
                                   (T)1, (T)2, l < L - 1, (T*)t.vin[l + 1], (T*)t.hpre[0], st));
    }
    // gh = gv * act'(h)
    act_bwd_kernel<T><<<ceil_div(pts * C, 256), 256, 0, st>>>(pts * C, gv, hpre, l < L - 1, gh);
    FCGNO_LAUNCHED();
    // pointwise weight and bias
    FCGNO_TRY(outer_reduce<T>(pts, C, C, gh, (const T*)t.vin[l], (T*)t.partials, grad + BL.w[l], grad + BL.b[l], st));
    // spectral: g' = w(k2) * sum_x gh e^{-i theta}  (analysis without 1/n, weights 1 / 2)
    Cx<T>* gspec = (Cx<T>*)s.spec2;
    FCGNO_TRY(launch_analysis<T>(N, B, C, M, nullptr, gh, (Cx<T>*)s.mid, gspec, (T)1, (T)2, tw1, tw2, st));
    spectral_wgrad_kernel<T, Gr><<<nmodes, 256, 0, st>>>(B, C, nmodes, (const Cx<T>*)t.chat[l], gspec, grad + BL.r[l]);
    FCGNO_LAUNCHED();
    // gc = R^H g'
    mix_kernel<T><<<nmodes, 256, C * C * sizeof(Cx<T>), st>>>(B, C, nmodes, nullptr, gspec, W.r[l], (Cx<T>*)s.spec, 1);
    FCGNO_LAUNCHED();
    // gv_in = W^T gh + (1/n) Re sum_k gc e^{+i theta}
    FCGNO_TRY(launch_synthesis_p<T>(N, B, C, M, nullptr, (Cx<T>*)s.spec, tw1, (Cx<T>*)s.mid, st));
    T* gnew = (gv == (T*)t.g0) ? (T*)t.gtmp : (T*)t.g0;  // ga (gtmp) is dead after the decoder
    FCGNO_TRY(launch_syn_q_pw<T>(N, B, C, M, nullptr, gh, (Cx<T>*)s.mid, tw2, W.w[l], 1, nullptr, inv_n, inv_n, 0,
                                 gnew, nullptr, st));
    gv = gnew;
  }
  // lift: A = gv0 [pts][C], V = x0 [pts][2]
  FCGNO_TRY(outer_reduce<T>(pts, C, 2, gv, (const T*)t.x0, (T*)t.partials, grad + BL.lift_w, grad + BL.lift_b, st));
  return FCGNO_OK;
}

// The BF16 training step: the Fourier layers forward and backward on the tensor cores (BF16
// operands, FP32 accumulation), everything else in FP32 on CUDA cores from the FP32 master
// weights (encoder, decoder, loss in FP64, every weight-gradient reduction).
static fcgno_status train_impl_tc(fcgno_model* m, fcgno_op* op, const double* r, const double* e, float* loss,
                                  float* grad, bool l2, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  const int B = op->B, C = d.width, M = d.modes, L = d.layers;
  const size_t n = op->n, pts = (size_t)B * n;
  const int nmodes = 2 * M * M;
  FCGNO_TRY(ensure_train(m, op, sizeof(float), true));
  TrainBuffers& t = m->ws->tr;
  Wp<float> W = wptrs<float>(m, m->w32);
  BlobLayout BL = blob_layout(d);
  FCGNO_TRY(tc_train_begin(m, op, st));
  FCGNO_TRY(launch_rms(r, B, n, t.rms, st));
  // the encoder's input x0 = (r / rms, log k) and its FP32 output, for the encoder's and the
  // first layer's weight gradients
  lift_kernel<float><<<dim3(ceil_div(n, 256), B), 256, 0, st>>>(B, n, C, r, op->logk, t.rms, nullptr, W.lift_w,
                                                                W.lift_b, (float*)t.vin[0], (float*)t.x0);
  FCGNO_LAUNCHED();
  float* cx[16];
  for (int l = 0; l < L; ++l) cx[l] = (float*)t.chat[l];
  FCGNO_TRY(tc_train_forward(m, op, r, t.rms, cx, st));
  for (int l = 1; l <= L; ++l) FCGNO_TRY(tc_train_to_f32(m, op, l, (float*)t.vin[l], st));
  const size_t smem = (size_t)d.proj_width * C * sizeof(float);
  project_kernel<float><<<dim3(ceil_div(n, 128), B), 128, smem, st>>>(
      n, C, d.proj_width, nullptr, (const float*)t.vin[L], W.proj1_w, W.proj1_b, W.proj2_w, W.proj2_b, t.rms,
      1.0 / ((double)(op->N + 1) * (op->N + 1)), d.output_scale ? op->kinv : nullptr, t.zbuf, (float*)t.apre,
      (float*)t.ghid, nullptr);
  FCGNO_LAUNCHED();
  FCGNO_TRY((loss_and_decoder_bwd<float, float>(m, op, e, loss, grad, l2, (const float*)t.vin[L], W, st)));
  float* gh = (float*)t.g1;
  for (int l = L - 1; l >= 0; --l) {
    FCGNO_TRY(tc_train_recompute_layer(m, op, l, st));
    FCGNO_TRY(tc_train_act_bwd(m, op, l, l == L - 1 ? (const float*)t.g0 : nullptr, gh, st));
    FCGNO_TRY(outer_reduce<float>(pts, C, C, gh, (const float*)t.vin[l], (float*)t.partials, grad + BL.w[l],
                                  grad + BL.b[l], st));
    FCGNO_TRY(tc_train_layer_bwd(m, op, l, st));
    spectral_wgrad_kernel<float, float><<<nmodes, 256, 0, st>>>(B, C, nmodes, (const Cx<float>*)t.chat[l],
                                                         (const Cx<float>*)tc_train_gspec(op), grad + BL.r[l]);
    FCGNO_LAUNCHED();
  }
  // encoder: A = gv0 [pts][C], V = x0 [pts][2]
  FCGNO_TRY(tc_train_to_f32(m, op, -1, (float*)t.g0, st));
  FCGNO_TRY(outer_reduce<float>(pts, C, 2, (const float*)t.g0, (const float*)t.x0, (float*)t.partials,
                                grad + BL.lift_w, grad + BL.lift_b, st));
  return FCGNO_OK;
}

fcgno_status train_step_simt(fcgno_model* m, fcgno_op* op, const double* r, const double* e, float* loss,
                             float* grad, fcgno_prec prec, bool l2, cudaStream_t st) {
  if (m->desc.width > 32 || m->desc.proj_width > 32 || 256 % m->desc.width != 0) {
    set_last_error("training supports width and proj_width <= 32 dividing 256");
    return FCGNO_EINVAL;
  }
  if (!m->ws) m->ws = new NoWorkspace();
  if (prec == FCGNO_BF16) return train_impl_tc(m, op, r, e, loss, grad, l2, st);
  if (prec == FCGNO_FP64) return train_impl<double, float>(m, op, r, e, loss, grad, l2, st);
  return train_impl<float, float>(m, op, r, e, loss, grad, l2, st);
}

fcgno_status train_step_f64(fcgno_model* m, fcgno_op* op, const double* r, const double* e, double* loss,
                            double* grad, bool l2, cudaStream_t st) {
  if (m->desc.width > 32 || m->desc.proj_width > 32 || 256 % m->desc.width != 0) {
    set_last_error("training supports width and proj_width <= 32 dividing 256");
    return FCGNO_EINVAL;
  }
  if (!m->ws) m->ws = new NoWorkspace();
  return train_impl<double, double>(m, op, r, e, loss, grad, l2, st);
}

}  // namespace fcgno
