// Fourier neural operator preconditioner on tcgen05 tensor cores (BF16 or FP16 operands,
// FP32 accumulation in tensor memory), Section 2.4.2 and Appendix A.
//
// Every contraction of a Fourier layer runs as a tcgen05.mma with operands staged in shared
// memory (no-swizzle core-matrix layouts) and the accumulator in TMEM:
//   analysis  stage Q : Z[(p,c)][(k2,t)]  = sum_q  v[q][p][c] E2[(k2,t)][q]     (A MN-major)
//   analysis  stage P : c[(k2,c)][(j,t')] = sum_(p,t) Z[(k2,c)][(p,t)] G[(j,t')][(p,t)]
//   mode mixing       : c'[b][(o,t')]     = sum_(i,t) c[b][(i,t)] Rr[(o,t')][(i,t)]   (per mode)
//   synthesis stage 1 : U[(k2,c)][(p,t')] = sum_(j,t) c'[(k2,c)][(j,t)] H[(p,t')][(j,t)]
//   synthesis stage 2 + pointwise, per tile of 128 grid points:
//       h[x][c] = sum_c' v[x][c'] W[c][c'] + sum_(pl,k2,t') Asyn[x][(pl,k2,t')] U[c][(pl,k2,t')]
//     (Asyn is block diagonal over the tile's grid columns when N < 128), then bias, GELU;
//     the last layer also runs the decoder C -> C_p (second MMA), GELU, -> 1, times h^2 rms(r).
// Tables: E2 = (cos, -sin)(2 pi k2 q / N); G = analysis twiddles over p with the 1/n factor;
// H = synthesis twiddles over p; Asyn = w_k2 (cos, -sin)(2 pi k2 q / N), w_0 = 1, w_{k2>0} = 2.
// Real and imaginary parts are interleaved along the contracted dimension, so every complex
// product is a real GEMM.
#include "internal.cuh"
#include "umma.cuh"

#include <vector>
#include <map>
#include <cmath>

namespace fcgno {

using namespace umma;

constexpr int kTcThreads = 128;

__device__ __forceinline__ uint16_t f2h16(float x, bool bf16) {
  if (bf16) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&h);
  }
  __half h = __float2half_rn(x);
  return *reinterpret_cast<uint16_t*>(&h);
}
__device__ __forceinline__ uint32_t pack2(float a, float b, bool bf16) {
  if (bf16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // one conversion for the pair
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// GELU of the 16-bit path in the tanh form of Hendrycks & Gimpel (2016),
// 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))), evaluated as x * sigmoid(2 sqrt(2/pi) (...))
// so that nothing cancels for negative x. It departs from the erf form by at most 4.7e-4
// (absolute), below the 16-bit rounding of the values it produces, and costs a few
// instructions instead of a branchy erf.
__device__ __forceinline__ float gelu16(float x) {
  const float u = 1.5957691216057308f * fmaf(0.044715f * x, x * x, x);
  return __fdividef(x, 1.0f + __expf(-u));
}

// Geometry shared by host and device.
struct TcGeom {
  int N, C, M, Ky, Kx4;   // Kx4 = 4M reals per (k2, c) row of mixed coefficients
  int KXP;                // Kx4 padded to 16
  int NPM;                // rows of G (= Kx4 padded to 16): N dimension of analysis stage P
  int MP;                 // Ky*C padded to 128
  int PC;                 // grid columns per analysis block (partial-sum chunk)
  int nchunks;            // N / PC
  int SPC;                // grid columns per synthesis block
  int snchunks;           // N / SPC
  int QC;                 // q rows per analysis K chunk
  int PT, QT;             // synthesis tile: PT columns x QT rows (= 128 points)
  int KSYN;               // K of the synthesis-stage-2 part, padded to 16
  int KB;                 // K extent of the staged U columns for one chunk (+16 zero pad)
  int nmodes;
};

static TcGeom make_geom(int N, int C, int M) {
  TcGeom g{};
  g.N = N;
  g.C = C;
  g.M = M;
  g.Ky = M;
  g.Kx4 = 4 * M;
  g.KXP = round_up(4 * M, 16);
  g.NPM = round_up(4 * M, 16);
  g.MP = round_up(M * C, 128);
  g.PC = N < 32 ? N : 32;
  // the synthesis stage-1 accumulator (MP/128 tiles x 2PC columns) must fit the 256 TMEM
  // columns a block allocates (two blocks share an SM's 512 columns)
  while ((g.MP / 128) * 2 * g.PC > 256 && g.PC > 8) g.PC /= 2;
  g.nchunks = N / g.PC;
  g.QC = N < 64 ? N : 64;
  if (N < 128) {
    g.PT = 128 / N;
    g.QT = N;
    g.KSYN = round_up(g.PT * 2 * M, 16);
  } else {
    g.PT = 1;
    g.QT = 128;
    g.KSYN = round_up(2 * M, 16);
  }
  // synthesis: narrower column chunks (more, smaller blocks; lower latency per instance)
  g.SPC = g.PC < 16 ? g.PC : 16;
  while (g.SPC % g.PT != 0) g.SPC *= 2;
  g.snchunks = N / g.SPC;
  g.KB = round_up(g.SPC * 2 * M, 16) + 16;
  g.nmodes = 2 * M * M;
  return g;
}

static bool geom_supported(int N, int C, int M, int Cp) {
  if (!(C == 16 || C == 32) || Cp != C || M < 1 || M > 16 || N < 2 * M) return false;
  if (!(N == 32 || N == 64 || (N >= 128 && N % 128 == 0))) return false;
  if ((std::min(N, 32) * C) % 128 != 0) return false;
  return true;
}

// ------------------------------------ tables -------------------------------------------
struct TcTables {
  int N = 0, M = 0;
  uint16_t* E2 = nullptr;    // [32][N]
  uint16_t* G = nullptr;     // [NPM][2N]
  uint16_t* H = nullptr;     // [2N][KXP]
  uint16_t* Asyn = nullptr;  // [rows][KSYN], rows = 128 (N < 128) or N
};

__device__ __forceinline__ void cs_of(long long k, long long x, int N, float& c, float& s) {
  const long long ph = ((k % N + N) % N) * x % N;
  double sd, cd;
  sincospi(2.0 * (double)ph / (double)N, &sd, &cd);
  c = (float)cd;
  s = (float)sd;
}

__global__ void tc_tables_kernel(TcGeom g, bool bf16, uint16_t* E2, uint16_t* G, uint16_t* H, uint16_t* Asyn) {
  const int N = g.N, M = g.M, Ky = g.Ky;
  const float inv_n = 1.0f / ((float)N * (float)N);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  // E2 [32][N]
  if (tid < 32 * N) {
    const int row = tid / N, q = tid % N, k2 = row >> 1, t = row & 1;
    float v = 0.f;
    if (k2 < Ky) {
      float c, s;
      cs_of(k2, q, N, c, s);
      v = t ? -s : c;
    }
    E2[tid] = f2h16(v, bf16);
  }
  // G [NPM][2N]
  if (tid < g.NPM * 2 * N) {
    const int row = tid / (2 * N), k = tid % (2 * N);
    const int j = row >> 1, tp = row & 1, p = k >> 1, t = k & 1;
    float v = 0.f;
    if (row < g.Kx4) {
      const int k1 = j < M ? j : j - 2 * M;
      float c, s;
      cs_of(k1, p, N, c, s);
      if (tp == 0) v = t == 0 ? c : s;
      else v = t == 0 ? -s : c;
      v *= inv_n;
    }
    G[tid] = f2h16(v, bf16);
  }
  // H [2N][KXP]
  if (tid < 2 * N * g.KXP) {
    const int row = tid / g.KXP, k = tid % g.KXP;
    const int p = row >> 1, tp = row & 1, j = k >> 1, t = k & 1;
    float v = 0.f;
    if (k < g.Kx4) {
      const int k1 = j < M ? j : j - 2 * M;
      float c, s;
      cs_of(k1, p, N, c, s);
      if (tp == 0) v = t == 0 ? c : -s;
      else v = t == 0 ? s : c;
    }
    H[tid] = f2h16(v, bf16);
  }
  // Asyn
  const int arows = N < 128 ? 128 : N;
  if (tid < arows * g.KSYN) {
    const int m = tid / g.KSYN, k = tid % g.KSYN;
    float v = 0.f;
    int pl, q;
    if (N < 128) {
      pl = m / N;
      q = m % N;
    } else {
      pl = 0;
      q = m;
    }
    const int pk = k / (2 * Ky), rem = k % (2 * Ky), k2 = rem >> 1, t = rem & 1;
    if (pl < g.PT && pk == pl && k < g.PT * 2 * Ky) {
      float c, s;
      cs_of(k2, q, N, c, s);
      const float w = k2 == 0 ? 1.f : 2.f;
      v = w * (t == 0 ? c : -s);
    }
    Asyn[tid] = f2h16(v, bf16);
  }
}

// ------------------------------------ model copies -------------------------------------
struct TcPrecision {
  bool built = false;
  std::vector<uint16_t*> W;   // [L] C x C
  std::vector<uint16_t*> Rr;  // [L] nmodes x 2C x 2C
  uint16_t* P1 = nullptr;     // Cp x C
  std::map<int, TcTables> tables;
};

}  // namespace fcgno

struct fcgno::TcModel {
  TcPrecision prec[2];  // 0: BF16, 1: FP16
  // activation workspace
  size_t cap_v = 0, cap_part = 0, cap_chat = 0;
  uint16_t* va = nullptr;
  uint16_t* vb = nullptr;
  float* part = nullptr;
  uint16_t* chat = nullptr;
};

namespace fcgno {

__global__ void tc_cast_kernel(size_t n, const float* __restrict__ in, uint16_t* __restrict__ out, bool bf16) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = f2h16(in[i], bf16);
}

// Rr[mode][(o,t')][(i,t)] from R[mode][i][o][re/im]
__global__ void tc_rr_kernel(int C, int nmodes, const float* __restrict__ R, uint16_t* __restrict__ Rr, bool bf16) {
  const size_t total = (size_t)nmodes * 4 * C * C;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int C2 = 2 * C;
  const size_t mode = idx / (C2 * C2);
  const int rem = (int)(idx % (C2 * C2));
  const int row = rem / C2, col = rem % C2;
  const int o = row >> 1, tp = row & 1, i = col >> 1, t = col & 1;
  const float re = R[((mode * C + i) * C + o) * 2], im = R[((mode * C + i) * C + o) * 2 + 1];
  float v;
  if (tp == 0) v = t == 0 ? re : -im;
  else v = t == 0 ? im : re;
  Rr[idx] = f2h16(v, bf16);
}

static void free_prec(TcPrecision& p) {
  for (auto x : p.W) cudaFree(x);
  for (auto x : p.Rr) cudaFree(x);
  p.W.clear();
  p.Rr.clear();
  if (p.P1) cudaFree(p.P1);
  p.P1 = nullptr;
  for (auto& kv : p.tables) {
    cudaFree(kv.second.E2);
    cudaFree(kv.second.G);
    cudaFree(kv.second.H);
    cudaFree(kv.second.Asyn);
  }
  p.tables.clear();
  p.built = false;
}

void tc_model_free(fcgno_model* m) {
  if (!m->tc) return;
  for (auto& p : m->tc->prec) free_prec(p);
  uint16_t* f[] = {m->tc->va, m->tc->vb, m->tc->chat};
  for (auto x : f)
    if (x) cudaFree(x);
  if (m->tc->part) cudaFree(m->tc->part);
  delete m->tc;
  m->tc = nullptr;
}

fcgno_status tc_model_sync(fcgno_model* m, cudaStream_t) {
  // weights changed: drop derived copies; they are rebuilt on next use
  m->gen++;
  if (m->tc)
    for (auto& p : m->tc->prec) {
      for (auto x : p.W) cudaFree(x);
      for (auto x : p.Rr) cudaFree(x);
      p.W.clear();
      p.Rr.clear();
      if (p.P1) cudaFree(p.P1);
      p.P1 = nullptr;
      p.built = false;
    }
  return FCGNO_OK;
}

static fcgno_status ensure_prec(fcgno_model* m, bool fp16, cudaStream_t st) {
  if (!m->tc) m->tc = new TcModel();
  TcPrecision& P = m->tc->prec[fp16 ? 1 : 0];
  if (P.built) return FCGNO_OK;
  const fcgno_model_desc& d = m->desc;
  const int C = d.width, Cp = d.proj_width, M = d.modes, nmodes = 2 * M * M;
  BlobLayout BL = blob_layout(d);
  const bool bf16 = !fp16;
  P.W.assign(d.layers, nullptr);
  P.Rr.assign(d.layers, nullptr);
  for (int l = 0; l < d.layers; ++l) {
    FCGNO_CUDA_TRY(cudaMalloc(&P.W[l], sizeof(uint16_t) * C * C));
    FCGNO_CUDA_TRY(cudaMalloc(&P.Rr[l], sizeof(uint16_t) * (size_t)nmodes * 4 * C * C));
    tc_cast_kernel<<<ceil_div(C * C, 256), 256, 0, st>>>(C * C, m->w32 + BL.w[l], P.W[l], bf16);
    FCGNO_LAUNCHED();
    const size_t tot = (size_t)nmodes * 4 * C * C;
    tc_rr_kernel<<<ceil_div(tot, 256), 256, 0, st>>>(C, nmodes, m->w32 + BL.r[l], P.Rr[l], bf16);
    FCGNO_LAUNCHED();
  }
  FCGNO_CUDA_TRY(cudaMalloc(&P.P1, sizeof(uint16_t) * Cp * C));
  tc_cast_kernel<<<ceil_div(Cp * C, 256), 256, 0, st>>>(Cp * C, m->w32 + BL.proj1_w, P.P1, bf16);
  FCGNO_LAUNCHED();
  P.built = true;
  m->gen++;
  return FCGNO_OK;
}

static fcgno_status ensure_tables(fcgno_model* m, bool fp16, const TcGeom& g, TcTables*& out, cudaStream_t st) {
  TcPrecision& P = m->tc->prec[fp16 ? 1 : 0];
  auto it = P.tables.find(g.N);
  if (it != P.tables.end() && it->second.M == g.M) {
    out = &it->second;
    return FCGNO_OK;
  }
  TcTables t;
  t.N = g.N;
  t.M = g.M;
  const int arows = g.N < 128 ? 128 : g.N;
  FCGNO_CUDA_TRY(cudaMalloc(&t.E2, sizeof(uint16_t) * 32 * g.N));
  FCGNO_CUDA_TRY(cudaMalloc(&t.G, sizeof(uint16_t) * g.NPM * 2 * g.N));
  FCGNO_CUDA_TRY(cudaMalloc(&t.H, sizeof(uint16_t) * 2 * g.N * g.KXP));
  FCGNO_CUDA_TRY(cudaMalloc(&t.Asyn, sizeof(uint16_t) * arows * g.KSYN));
  const int work = std::max(std::max(32 * g.N, g.NPM * 2 * g.N), std::max(2 * g.N * g.KXP, arows * g.KSYN));
  tc_tables_kernel<<<ceil_div(work, 256), 256, 0, st>>>(g, !fp16, t.E2, t.G, t.H, t.Asyn);
  FCGNO_LAUNCHED();
  P.tables[g.N] = t;
  out = &P.tables[g.N];
  m->gen++;
  return FCGNO_OK;
}

// ------------------------------------ kernels ------------------------------------------
__device__ __forceinline__ bool tc_inactive(const int* active, int b) { return active && active[b] >= 0; }

// Encoder: v0 = lift_w [r/rms, log k] + lift_b, written as 16-bit channels-last. One thread
// per grid point; the only FP64 work is reading r (1/rms is formed once per thread in FP32).
template <int C>
__global__ void tc_lift_kernel(size_t n, const double* __restrict__ r, const float* __restrict__ logk,
                               const double* __restrict__ rms, const int* __restrict__ active,
                               const float* __restrict__ lw, const float* __restrict__ lb, uint16_t* __restrict__ v,
                               bool bf16) {
  __shared__ float w0[C], w1[C], bb[C];
  const int b = blockIdx.y;
  if (tc_inactive(active, b)) return;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    w0[c] = lw[2 * c];
    w1[c] = lw[2 * c + 1];
    bb[c] = lb[c];
  }
  __syncthreads();
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= n) return;
  const float s = (float)rms[b];
  const float inv = s > 0.f ? 1.0f / s : 0.f;
  const float rh = (float)r[(size_t)b * n + x] * inv;
  const float lk = logk[(size_t)b * n + x];
  uint4* dst = reinterpret_cast<uint4*>(v + ((size_t)b * n + x) * C);
#pragma unroll
  for (int c0 = 0; c0 < C; c0 += 8) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = c0 + 2 * i;
      w[i] = pack2(fmaf(w0[c], rh, fmaf(w1[c], lk, bb[c])), fmaf(w0[c + 1], rh, fmaf(w1[c + 1], lk, bb[c + 1])), bf16);
    }
    dst[c0 / 8] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Truncated analysis of one grid-column chunk of one instance; writes FP32 partial sums
// part[b][chunk][mode = j*Ky + k2][c][re/im].
template <int C>
__global__ void __launch_bounds__(kTcThreads, 2)
    tc_analysis_kernel(TcGeom g, bool bf16, const int* __restrict__ active, const uint16_t* __restrict__ v,
                       const uint16_t* __restrict__ E2, const uint16_t* __restrict__ G, float* __restrict__ part,
                       int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t mbar, mbar2[3];
  __shared__ uint32_t tbase_s;
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (tc_inactive(active, b)) return;
  const int N = g.N, PC = g.PC, QC = g.QC, Ky = g.Ky;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // shared layout
  const int ne2 = (N / QC > 1) ? 3 : 1;             // E2 changes per q chunk only when N > QC
  uint8_t* sE2 = smem;                              // ne2 x (32 x QC), K-major: LBO 128, SBO QC*16
  uint8_t* sA = sE2 + ne2 * 32 * QC * 2;            // 3 x (128 x QC), MN-major: SBO 128, LBO 2048
  uint8_t* sAP = sA + 3 * 128 * QC * 2;             // MP x 2PC, K-major: LBO 128, SBO 2PC*16
  uint8_t* sG = sAP + (size_t)g.MP * 2 * PC * 2;    // NPM x 2PC, K-major: LBO 128, SBO 2PC*16
  const uint32_t SBO_E = QC * 16, SBO_P = 2 * PC * 16, SBO_G = 2 * PC * 16;
  const uint32_t LBO_A = 2048;  // k-direction stride of the MN-major stage-Q operand (16 m-core matrices)

  const uint32_t tcols = (64 + (g.MP / 128) * g.NPM) <= 256 ? 256u : 512u;
  if (warp == 0) tmem_alloc(&tbase_s, tcols);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    mbar_init(&mbar2[0], 1);
    mbar_init(&mbar2[1], 1);
    mbar_init(&mbar2[2], 1);
  }
  // stage G slice (k = 2*p0 .. 2*p0 + 2PC) and zero the padding rows of sAP
  const int p0 = chunk * PC;
  for (int idx = tid; idx < g.NPM * (2 * PC / 8); idx += kTcThreads) {
    const int row = idx / (2 * PC / 8), kc = idx % (2 * PC / 8);
    const uint4 val = *reinterpret_cast<const uint4*>(G + (size_t)row * 2 * N + 2 * p0 + kc * 8);
    *reinterpret_cast<uint4*>(sG + kmajor_off(row, kc * 8, 128, SBO_G)) = val;
  }
  for (int idx = tid; idx < (g.MP - Ky * C) * (2 * PC / 8); idx += kTcThreads) {
    const int row = Ky * C + idx / (2 * PC / 8), kc = idx % (2 * PC / 8);
    *reinterpret_cast<uint4*>(sAP + kmajor_off(row, kc * 8, 128, SBO_P)) = make_uint4(0, 0, 0, 0);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tbase_s;
  const uint32_t tQ = tbase, tP = tbase + 64;  // two Z slots of 32 columns, then the c accumulators
  uint32_t phase = 0;
  bool ok = true;
  const uint16_t* vb = v + (size_t)b * N * N * C;
  const int mtiles = PC * C / 128;
  const int qchunks = N / QC;
  constexpr uint32_t idQ = idesc_f16(128, 32, true, true, false);
  constexpr uint32_t idQh = idesc_f16(128, 32, false, true, false);
  // Steps s = (m-tile, q-chunk) run through a three-slot pipeline: while the MMA of step s
  // runs, the operands of steps s+1 and s+2 are in flight; the Z accumulator alternates
  // between two TMEM slots by m-tile so that the read-back of one m-tile overlaps the MMAs
  // of the next.
  constexpr int NS = 3;
  const int nsteps = mtiles * qchunks;
  uint32_t phs[NS] = {0, 0, 0};
  bool pending[NS] = {false, false, false};
  auto stage = [&](int st_, int buf) {
    const int mt = st_ / qchunks, qc = st_ % qchunks, q0 = qc * QC;
    if (qchunks > 1 || st_ == 0) {
      uint8_t* e2 = sE2 + (qchunks > 1 ? buf * 32 * QC * 2 : 0);
      for (int idx = tid; idx < 32 * (QC / 8); idx += kTcThreads) {
        const int row = idx / (QC / 8), kc = idx % (QC / 8);
        cp_async16(e2 + kmajor_off(row, kc * 8, 128, SBO_E), E2 + (size_t)row * N + q0 + kc * 8);
      }
    }
    // A tile: m = local (p, c) index 128*mt .. +128, k = q: 16-byte runs of 8 channels
    uint8_t* sa = sA + buf * 128 * QC * 2;
    for (int idx = tid; idx < QC * 16; idx += kTcThreads) {
      const int ql = idx >> 4, mc = idx & 15;  // mc: 8-channel group within the 128 rows
      const int m = mt * 128 + mc * 8;
      const int pl = m / C, c0 = m % C;
      cp_async16(sa + mnmajor_off(mc * 8, ql, LBO_A, 128), vb + ((size_t)(q0 + ql) * N + (p0 + pl)) * C + c0);
    }
    cp_async_commit();
  };
  auto wait_slot = [&](int buf) -> bool {
    if (!pending[buf]) return true;
    const bool r = mbar_wait(&mbar2[buf], phs[buf]);
    phs[buf] ^= 1;
    pending[buf] = false;
    fence_after_sync();
    return r;
  };
  stage(0, 0);
  if (nsteps > 1) stage(1, 1);
  for (int st_ = 0; st_ < nsteps && ok; ++st_) {
    const int buf = st_ % NS, mt = st_ / qchunks, qc = st_ % qchunks;
    if (st_ + 1 < nsteps)
      cp_async_wait_all_but_one();  // step st_'s copies done, step st_+1's may still fly
    else
      cp_async_wait_all();
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tq = tQ + (mt & 1) * 32;
    if (tid == 0) {
      const uint32_t sa = smem_addr(sA + buf * 128 * QC * 2);
      const uint32_t e2 = smem_addr(sE2 + (qchunks > 1 ? buf * 32 * QC * 2 : 0));
      for (int ks = 0; ks < QC / 16; ++ks)
        mma(tq, desc(sa + ks * 2 * LBO_A, LBO_A, 128), desc(e2 + ks * 2 * 128, 128, SBO_E), bf16 ? idQ : idQh,
            qc > 0 || ks > 0);
      commit(&mbar2[buf]);
    }
    pending[buf] = true;
    if (st_ + 2 < nsteps) {
      // the slot of step st_-1: its MMA must have finished before it is refilled
      const int nb = (st_ + 2) % NS;
      ok = wait_slot(nb);
      if (!ok) break;
      stage(st_ + 2, nb);
    }
    if (qc == qchunks - 1) {
      ok = wait_slot(buf);
      if (!ok) break;
      // read Z for this m-tile: lane = (p, c), columns (k2, t) -> sAP[(k2, c)][(p, t)]
      const int m = mt * 128 + warp * 32 + lane;
      const int pl = m / C, c = m % C;
      float z[32];
      float tmp[16];
      tmem_ld16(tq + ((uint32_t)(warp * 32) << 16), tmp);
#pragma unroll
      for (int i = 0; i < 16; ++i) z[i] = tmp[i];
      tmem_ld16(tq + ((uint32_t)(warp * 32) << 16) + 16, tmp);
#pragma unroll
      for (int i = 0; i < 16; ++i) z[16 + i] = tmp[i];
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {  // Ky <= 16: static indices keep z in registers
        if (k2 < Ky) {
          const int row = k2 * C + c;
          *reinterpret_cast<uint32_t*>(sAP + kmajor_off(row, 2 * pl, 128, SBO_P)) =
              pack2(z[2 * k2], z[2 * k2 + 1], bf16);
        }
      }
    }
  }
  cp_async_wait_all();
  if (ok) {
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const int ptiles = g.MP / 128;
    if (tid == 0) {
      const uint32_t id = idesc_f16(128, g.NPM, bf16, false, false);
      for (int pt = 0; pt < ptiles; ++pt)
        for (int ks = 0; ks < 2 * PC / 16; ++ks) {
          const uint64_t ad = desc(smem_addr(sAP) + pt * 16 * SBO_P + ks * 2 * 128, 128, SBO_P);
          const uint64_t bd = desc(smem_addr(sG) + ks * 2 * 128, 128, SBO_G);
          mma(tP + pt * g.NPM, ad, bd, id, ks > 0);
        }
      commit(&mbar);
    }
    ok = mbar_wait(&mbar, phase);
    phase ^= 1;
    fence_after_sync();
    if (ok) {
      float* pb = part + ((size_t)b * g.nchunks + chunk) * g.nmodes * C * 2;
      for (int pt = 0; pt < ptiles; ++pt) {
        const int row = pt * 128 + warp * 32 + lane;
        const int k2 = row / C, c = row % C;
        for (int c0 = 0; c0 < g.NPM; c0 += 16) {
          float val[16];
          tmem_ld16(tP + pt * g.NPM + c0 + ((uint32_t)(warp * 32) << 16), val);
          if (row < Ky * C) {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
              const int j = (c0 + i) >> 1;
              if (j < 2 * g.M) {
                float2 w2 = make_float2(val[i], val[i + 1]);
                *reinterpret_cast<float2*>(pb + ((size_t)(j * Ky + k2) * C + c) * 2) = w2;
              }
            }
          }
        }
      }
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, tcols);
}

// Per-mode complex channel mixing across instances: rows = instances (128 per CTA).
// Output c'[b][(j, re/im)][(k2, c)] (16-bit): the MN-major layout of the synthesis stage-1
// A operand, so that each instance's C outputs of one (mode, re/im) are one 2C-byte run.
template <int C>
__global__ void __launch_bounds__(kTcThreads)
    tc_mix_kernel(TcGeom g, int B, bool bf16, const int* __restrict__ active, const float* __restrict__ part,
                  const uint16_t* __restrict__ Rr, uint16_t* __restrict__ chat, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase_s;
  __shared__ int any_active;
  constexpr int C2 = 2 * C;
  const int mode = blockIdx.x, b0 = blockIdx.y * 128;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) any_active = 0;
  __syncthreads();
  if (b0 + tid < B && !tc_inactive(active, b0 + tid)) any_active = 1;
  __syncthreads();
  if (!any_active) return;  // every instance of this tile has stopped
  uint8_t* sA = smem;              // 128 x C2, K-major, SBO = C2*16
  uint8_t* sB = sA + 128 * C2 * 2; // C2 x C2,  K-major
  constexpr uint32_t SBO = C2 * 16;
  if (warp == 0) tmem_alloc(&tbase_s, C2 < 32 ? 32 : C2);
  if (tid == 0) mbar_init(&mbar, 1);
  {
    // warp w loads rows 32w..32w+31; a row (one instance's C2 values) is one coalesced read
    // per chunk, the chunks are summed in order
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const int row = warp * 32 + r;
      const int b = b0 + row;
      float2 acc = make_float2(0.f, 0.f);
      if (b < B && 2 * lane < C2) {
        for (int ch = 0; ch < g.nchunks; ++ch) {
          const float2 v = *reinterpret_cast<const float2*>(part + (((size_t)b * g.nchunks + ch) * g.nmodes + mode) * C2 +
                                                            2 * lane);
          acc.x += v.x;
          acc.y += v.y;
        }
      }
      if (2 * lane < C2)
        *reinterpret_cast<uint32_t*>(sA + kmajor_off(row, 2 * lane, 128, SBO)) = pack2(acc.x, acc.y, bf16);
    }
    const uint16_t* Rm = Rr + (size_t)mode * C2 * C2;
    for (int idx = tid; idx < C2 * C2 / 8; idx += kTcThreads) {
      const int r = idx / (C2 / 8), kc = idx % (C2 / 8);
      cp_async16(sB + kmajor_off(r, kc * 8, 128, SBO), Rm + r * C2 + kc * 8);
    }
    cp_async_commit();
    cp_async_wait_all();
  }
  fence_smem_to_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tbase_s;
  if (tid == 0) {
    const uint32_t id = idesc_f16(128, C2, bf16, false, false);
    for (int ks = 0; ks < C2 / 16; ++ks)
      mma(tbase, desc(smem_addr(sA) + ks * 256, 128, SBO), desc(smem_addr(sB) + ks * 256, 128, SBO), id, ks > 0);
    commit(&mbar);
  }
  const bool ok = mbar_wait(&mbar, 0);
  fence_after_sync();
  if (ok) {
    const int b = b0 + warp * 32 + lane;
    const int j = mode / g.Ky, k2 = mode % g.Ky;
    float val[C2];
#pragma unroll
    for (int c0 = 0; c0 < C2; c0 += 16) {
      float t16[16];
      tmem_ld16(tbase + c0 + ((uint32_t)(warp * 32) << 16), t16);
#pragma unroll
      for (int i = 0; i < 16; ++i) val[c0 + i] = t16[i];
    }
    if (b < B) {
      // columns are (o, re/im) interleaved; write the C real parts, then the C imaginary parts
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        uint4* dst = reinterpret_cast<uint4*>(chat + (((size_t)b * g.Kx4 + 2 * j + t) * g.Ky + k2) * C);
#pragma unroll
        for (int o0 = 0; o0 < C; o0 += 8) {
          dst[o0 / 8] = make_uint4(pack2(val[2 * o0 + t], val[2 * o0 + 2 + t], bf16),
                                   pack2(val[2 * o0 + 4 + t], val[2 * o0 + 6 + t], bf16),
                                   pack2(val[2 * o0 + 8 + t], val[2 * o0 + 10 + t], bf16),
                                   pack2(val[2 * o0 + 12 + t], val[2 * o0 + 14 + t], bf16));
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, C2 < 32 ? 32 : C2);
}

struct SynArgs {
  TcGeom g;
  int B;
  bool bf16;
  const int* active;
  const uint16_t* chat;   // [B][Kx4][Ky][C]  (MN-major stage-1 operand)
  const uint16_t* vin;    // [B][N][N][C]
  const uint16_t* W;      // [C][C]
  const float* bias;      // [C]
  const uint16_t* H;      // [2N][KXP]
  const uint16_t* Asyn;   // [rows][KSYN]
  int activate;
  uint16_t* vout;         // [B][N][N][C] (hidden layers)
  // decoder (last layer)
  int project;
  const uint16_t* P1;     // [C][C]
  const float* p1;
  const float* p2;
  const float* p2b;
  const double* rms;
  double hh;              // h^2 output scale
  double* z;              // [B][N][N]
  int* err;
};

// Synthesis + pointwise + bias + activation (+ decoder) for one grid-column chunk of one instance.
template <int C>
__global__ void __launch_bounds__(kTcThreads, 2) tc_synthesis_kernel(SynArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t mbar[4];
  __shared__ uint32_t tbase_s;
  const TcGeom& g = a.g;
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (tc_inactive(a.active, b)) return;
  const int N = g.N, PC = g.SPC, Ky = g.Ky;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool bf16 = a.bf16;
  const int p0 = chunk * PC;
  // shared layout
  const uint32_t LBO_A1 = (g.MP / 8) * 128;  // MN-major: K-direction core-matrix stride
  const uint32_t SBO_H = g.KXP * 16, SBO_B = g.KB * 16, SBO_S = g.KSYN * 16, SBO_C = C * 16;
  // region R0 holds the mixed coefficients for synthesis stage 1, then (aliased, once stage 1
  // has completed) a ring of three pointwise input tiles, the decoder input tile and, for
  // N >= 128, the per-tile rows of the synthesis table
  const size_t TB = (size_t)128 * C * 2, SB = (size_t)128 * g.KSYN * 2;
  const size_t r0a = (size_t)g.MP * g.KXP * 2, r0b = 4 * TB + (N >= 128 ? 3 * SB : 0);
  const size_t r0 = r0a > r0b ? r0a : r0b;
  uint8_t* sA1 = smem;                                  // MP x KXP
  uint8_t* sX0 = smem;                                  // 3 x (128 x C) pointwise tiles (after stage 1)
  uint8_t* sD = smem + 3 * TB;                          // 128 x C decoder input (after stage 1)
  uint8_t* sSb = smem + 4 * TB;                         // 3 x (128 x KSYN) table rows (N >= 128)
  uint8_t* sH = smem + r0;                              // 2PC x KXP
  uint8_t* sB = sH + (size_t)2 * PC * g.KXP * 2;        // C x KB
  uint8_t* sS = sB + (size_t)C * g.KB * 2;              // 128 x KSYN (N < 128: one table for all tiles)
  uint8_t* sW = sS + (N < 128 ? SB : 0);                // C x C
  uint8_t* sP = sW + C * C * 2;                         // C x C (decoder)
  const uint32_t TCOLS = 256;
  if (warp == 0) tmem_alloc(&tbase_s, TCOLS);
  if (tid < 4) mbar_init(&mbar[tid], 1);
  // ---- stage operands that do not change across tiles
  // mixed coefficients, MN-major: element (m = (k2, c), k = (j, re/im)) is at
  // chat[b][k][m]; 8 consecutive m at one k form one 16-byte run
  const uint16_t* cb = a.chat + (size_t)b * g.Kx4 * Ky * C;
  for (int idx = tid; idx < (g.MP / 8) * g.KXP; idx += kTcThreads) {
    const int k = idx / (g.MP / 8), mc = idx % (g.MP / 8);
    uint8_t* dst = sA1 + mnmajor_off(mc * 8, k, LBO_A1, 128);
    if (mc * 8 < Ky * C && k < g.Kx4)
      cp_async16(dst, cb + (size_t)k * Ky * C + mc * 8);
    else
      *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
  }
  for (int idx = tid; idx < 2 * PC * (g.KXP / 8); idx += kTcThreads) {
    const int row = idx / (g.KXP / 8), kc = idx % (g.KXP / 8);
    cp_async16(sH + kmajor_off(row, kc * 8, 128, SBO_H), a.H + (size_t)(2 * p0 + row) * g.KXP + kc * 8);
  }
  for (int idx = tid; idx < C * (C / 8); idx += kTcThreads) {
    const int row = idx / (C / 8), kc = idx % (C / 8);
    *reinterpret_cast<uint4*>(sW + kmajor_off(row, kc * 8, 128, SBO_C)) =
        *reinterpret_cast<const uint4*>(a.W + row * C + kc * 8);
    if (a.project)
      *reinterpret_cast<uint4*>(sP + kmajor_off(row, kc * 8, 128, SBO_C)) =
          *reinterpret_cast<const uint4*>(a.P1 + row * C + kc * 8);
  }
  if (N < 128) {
    for (int idx = tid; idx < 128 * (g.KSYN / 8); idx += kTcThreads) {
      const int row = idx / (g.KSYN / 8), kc = idx % (g.KSYN / 8);
      cp_async16(sS + kmajor_off(row, kc * 8, 128, SBO_S), a.Asyn + (size_t)row * g.KSYN + kc * 8);
    }
  }
  cp_async_commit();
  // zero the K tail of the staged U columns (read by padded synthesis K steps)
  const int kvalid = PC * 2 * Ky;
  for (int idx = tid; idx < C * ((g.KB - (kvalid & ~7)) / 8); idx += kTcThreads) {
    const int nk = (g.KB - (kvalid & ~7)) / 8;
    const int row = idx / nk, kc = (kvalid & ~7) / 8 + idx % nk;
    *reinterpret_cast<uint4*>(sB + kmajor_off(row, kc * 8, 128, SBO_B)) = make_uint4(0, 0, 0, 0);
  }
  cp_async_wait_all();
  fence_smem_to_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tbase_s;
  const uint32_t tU = tbase;              // (MP/128) x 2PC columns (stage 1)
  const uint32_t tD = tbase;              // 2 x C tile accumulators (reuse U's columns after stage 1)
  const uint32_t tE = tbase + 2 * C;      // C decoder accumulator
  uint32_t ph[4] = {0, 0, 0, 0};
  bool ok = true;
  const int utiles = g.MP / 128;
  // ---- synthesis stage 1: U = c' H^T for the chunk
  if (tid == 0) {
    const uint32_t id = idesc_f16(128, 2 * PC, bf16, true, false);
    for (int ut = 0; ut < utiles; ++ut)
      for (int ks = 0; ks < g.KXP / 16; ++ks)
        mma(tU + ut * 2 * PC, desc(smem_addr(sA1) + ut * 16 * 128 + ks * 2 * LBO_A1, LBO_A1, 128),
            desc(smem_addr(sH) + ks * 256, 128, SBO_H), id, ks > 0);
    commit(&mbar[0]);
  }
  ok = mbar_wait(&mbar[0], ph[0]);
  ph[0] ^= 1;
  fence_after_sync();
  if (ok) {
    // U lane (k2, c), columns (p, t') -> sB[c][(p, k2, t')]
    for (int ut = 0; ut < utiles; ++ut) {
      const int row = ut * 128 + warp * 32 + lane;
      const int k2 = row / C, c = row % C;
      for (int c0 = 0; c0 < 2 * PC; c0 += 16) {
        float val[16];
        tmem_ld16(tU + ut * 2 * PC + c0 + ((uint32_t)(warp * 32) << 16), val);
        if (row < Ky * C) {
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const int pl = (c0 + i) >> 1;
            *reinterpret_cast<uint32_t*>(sB + kmajor_off(c, pl * 2 * Ky + 2 * k2, 128, SBO_B)) =
                pack2(val[i], val[i + 1], bf16);
          }
        }
      }
    }
  }
  fence_smem_to_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  // ---- tiles of 128 grid points
  const int ntiles = (N < 128) ? PC / g.PT : PC * (N / 128);
  const uint16_t* vb = a.vin + (size_t)b * N * N * C;
  // Thread tid owns tile row m = tid of every tile: its grid point within the tile is fixed,
  // so the row's (q, column offset) and shared-memory offsets are computed once.
  const int m_own = tid;
  const int own_pl = (N < 128) ? m_own / N : 0;     // column within the tile (N < 128)
  const int own_q = (N < 128) ? m_own % N : m_own;  // row (N < 128) or row within the q-tile
  const bool own_valid = (N < 128) ? own_pl < g.PT : true;
  const uint32_t own_xoff = kmajor_off(m_own, 0, 128, SBO_C);
  auto tile_point = [&](int t, int& q, int& p) {
    if (N < 128) {
      q = own_q;
      p = p0 + t * g.PT + own_pl;
    } else {
      const int col = t / (N / 128), qt = t % (N / 128);
      p = p0 + col;
      q = qt * 128 + own_q;
    }
  };
  auto prefetch = [&](int t, int buf) {
    uint8_t* dst = sX0 + buf * TB + own_xoff;
    int q, p;
    tile_point(t, q, p);
    const uint16_t* src = vb + ((size_t)q * N + p) * C;
#pragma unroll
    for (int kc = 0; kc < C / 8; ++kc) {
      if (own_valid)
        cp_async16(dst + kc * 128, src + kc * 8);
      else
        *reinterpret_cast<uint4*>(dst + kc * 128) = make_uint4(0, 0, 0, 0);
    }
    if (N >= 128) {
      // synthesis-table rows of this tile's q range, in the tile's ring slot
      const int qt = t % (N / 128);
      uint8_t* sdst = sSb + buf * SB;
      for (int idx = tid; idx < 128 * (g.KSYN / 8); idx += kTcThreads) {
        const int row = idx / (g.KSYN / 8), kc = idx % (g.KSYN / 8);
        cp_async16(sdst + kmajor_off(row, kc * 8, 128, SBO_S), a.Asyn + (size_t)(qt * 128 + row) * g.KSYN + kc * 8);
      }
    }
    cp_async_commit();
  };
  const uint32_t idD = idesc_f16(128, C, bf16);
  // tile t: ring slot t % 3, accumulator slot t % 2; issued by thread 0
  auto mma_tile = [&](int t) {
    const int buf = t % 3, acc = t & 1;
    const uint32_t sx = smem_addr(sX0 + buf * TB);
    const uint32_t ss = (N < 128) ? smem_addr(sS) : smem_addr(sSb + buf * SB);
    for (int ks = 0; ks < C / 16; ++ks)
      mma(tD + acc * C, desc(sx + ks * 256, 128, SBO_C), desc(smem_addr(sW) + ks * 256, 128, SBO_C), idD, ks > 0);
    const int kb0 = (N < 128) ? t * g.PT * 2 * Ky : (t / (N / 128)) * 2 * Ky;
    for (int ks = 0; ks < g.KSYN / 16; ++ks)
      mma(tD + acc * C, desc(ss + ks * 256, 128, SBO_S), desc(smem_addr(sB) + (kb0 / 8) * 128 + ks * 256, 128, SBO_B),
          idD, true);
    commit(&mbar[1 + acc]);
  };
  float bias[C];
#pragma unroll
  for (int c = 0; c < C; ++c) bias[c] = a.bias[c];
  // Software pipeline: while tile t's epilogue runs, tile t+1's MMA runs on the tensor core
  // (other accumulator) and tile t+2's operands are being copied (third ring slot).
  if (ok && ntiles > 0) {
    prefetch(0, 0);
    if (ntiles > 1) {
      prefetch(1, 1);
      cp_async_wait_all_but_one();
    } else {
      cp_async_wait_all();
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid == 0) mma_tile(0);
  }
  for (int t = 0; t < ntiles && ok; ++t) {
    if (t + 1 < ntiles) {
      cp_async_wait_all();  // tile t+1's copies (the only group in flight)
      fence_smem_to_async();
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (tid == 0) mma_tile(t + 1);
      // ring slot of tile t-1, whose MMA completed before its epilogue
      if (t + 2 < ntiles) prefetch(t + 2, (t + 2) % 3);
    }
    const int buf = t & 1;
    ok = mbar_wait(&mbar[1 + buf], ph[1 + buf]);
    ph[1 + buf] ^= 1;
    fence_after_sync();
    if (!ok) break;
    // epilogue: lane = grid point, C columns
    const int m = m_own;
    int q, p;
    tile_point(t, q, p);
    const bool valid = own_valid;
    float h[C];
#pragma unroll
    for (int c0 = 0; c0 < C; c0 += 16) {
      float val[16];
      tmem_ld16(tD + buf * C + c0 + ((uint32_t)(warp * 32) << 16), val);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float x = val[i] + bias[c0 + i];
        h[c0 + i] = a.activate ? gelu16(x) : x;
      }
    }
    if (!a.project) {
      if (valid) {
        uint16_t* dst = a.vout + (((size_t)b * N + q) * N + p) * C;
#pragma unroll
        for (int c0 = 0; c0 < C; c0 += 8) {
          uint4 w = make_uint4(pack2(h[c0], h[c0 + 1], bf16), pack2(h[c0 + 2], h[c0 + 3], bf16),
                               pack2(h[c0 + 4], h[c0 + 5], bf16), pack2(h[c0 + 6], h[c0 + 7], bf16));
          *reinterpret_cast<uint4*>(dst + c0) = w;
        }
      }
    } else {
      // decoder: second MMA on the 16-bit layer output
#pragma unroll
      for (int c0 = 0; c0 < C; c0 += 8) {
        uint4 w = make_uint4(pack2(h[c0], h[c0 + 1], bf16), pack2(h[c0 + 2], h[c0 + 3], bf16),
                             pack2(h[c0 + 4], h[c0 + 5], bf16), pack2(h[c0 + 6], h[c0 + 7], bf16));
        *reinterpret_cast<uint4*>(sD + kmajor_off(m, c0, 128, SBO_C)) = w;
      }
      fence_smem_to_async();
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (tid == 0) {
        for (int ks = 0; ks < C / 16; ++ks)
          mma(tE, desc(smem_addr(sD) + ks * 256, 128, SBO_C), desc(smem_addr(sP) + ks * 256, 128, SBO_C), idD, ks > 0);
        commit(&mbar[3]);
      }
      ok = mbar_wait(&mbar[3], ph[3]);
      ph[3] ^= 1;
      fence_after_sync();
      if (!ok) break;
      float zt = a.p2b[0];
#pragma unroll
      for (int c0 = 0; c0 < C; c0 += 16) {
        float val[16];
        tmem_ld16(tE + c0 + ((uint32_t)(warp * 32) << 16), val);
#pragma unroll
        for (int i = 0; i < 16; ++i) zt = fmaf(a.p2[c0 + i], gelu16(val[i] + a.p1[c0 + i]), zt);
      }
      if (valid) a.z[((size_t)b * N + q) * N + p] = a.rms[b] * a.hh * (double)zt;
    }
    fence_before_sync();
  }
  cp_async_wait_all();
  if (!ok && tid == 0) atomicExch(a.err, 1);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, TCOLS);
}

// ------------------------------------ host ---------------------------------------------
static size_t analysis_smem(const TcGeom& g) {
  const int ne2 = (g.N / g.QC > 1) ? 3 : 1;
  return (size_t)ne2 * 32 * g.QC * 2 + (size_t)3 * 128 * g.QC * 2 + (size_t)g.MP * 2 * g.PC * 2 +
         (size_t)g.NPM * 2 * g.PC * 2;
}
static size_t mix_smem(int C) { return (size_t)128 * 2 * C * 2 + (size_t)4 * C * C * 2; }
static size_t synthesis_smem(const TcGeom& g) {
  const int C = g.C;
  const size_t TB = (size_t)128 * C * 2, SB = (size_t)128 * g.KSYN * 2;
  const size_t r0 = std::max((size_t)g.MP * g.KXP * 2, 4 * TB + (g.N >= 128 ? 3 * SB : 0));
  return r0 + (size_t)2 * g.SPC * g.KXP * 2 + (size_t)C * g.KB * 2 + (g.N < 128 ? SB : 0) + (size_t)2 * C * C * 2;
}

template <int C>
static fcgno_status run_tc(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms, const int* active,
                           double* z, bool fp16, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  const TcGeom g = make_geom(op->N, C, d.modes);
  FCGNO_TRY(ensure_prec(m, fp16, st));
  TcTables* tab = nullptr;
  FCGNO_TRY(ensure_tables(m, fp16, g, tab, st));
  TcModel& T = *m->tc;
  TcPrecision& P = T.prec[fp16 ? 1 : 0];
  const int B = op->B;
  const size_t n = op->n;
  const size_t need_v = (size_t)B * n * C, need_part = (size_t)B * g.nchunks * g.nmodes * C * 2,
               need_chat = (size_t)B * g.Ky * C * g.Kx4;
  if (T.cap_v < need_v || T.cap_part < need_part || T.cap_chat < need_chat) {
    if (T.va) cudaFree(T.va);
    if (T.vb) cudaFree(T.vb);
    if (T.part) cudaFree(T.part);
    if (T.chat) cudaFree(T.chat);
    T.va = T.vb = T.chat = nullptr;
    T.part = nullptr;
    T.cap_v = T.cap_part = T.cap_chat = 0;
    if (cudaMalloc(&T.va, need_v * 2) != cudaSuccess || cudaMalloc(&T.vb, need_v * 2) != cudaSuccess ||
        cudaMalloc(&T.part, need_part * 4) != cudaSuccess || cudaMalloc(&T.chat, need_chat * 2) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("tensor-core preconditioner workspace: out of device memory");
      return FCGNO_ENOMEM;
    }
    T.cap_v = need_v;
    T.cap_part = need_part;
    T.cap_chat = need_chat;
    m->gen++;
  }
  static int* d_err = nullptr;
  if (!d_err) {
    FCGNO_CUDA_TRY(cudaMalloc(&d_err, sizeof(int)));
    FCGNO_CUDA_TRY(cudaMemset(d_err, 0, sizeof(int)));
  }
  BlobLayout BL = blob_layout(d);
  const bool bf16 = !fp16;
  {
    TraceScope ts("tc_lift", st);
    tc_lift_kernel<C><<<dim3(ceil_div(n, 256), B), 256, 0, st>>>(n, r, op->logk32, rms, active, m->w32 + BL.lift_w,
                                                                 m->w32 + BL.lift_b, T.va, bf16);
  }
  FCGNO_LAUNCHED();
  const size_t sa = analysis_smem(g), ss = synthesis_smem(g), sm = mix_smem(C);
  // raise the dynamic shared-memory limit only when a larger plan appears (not a stream
  // operation; the first solve iteration runs eagerly, before any graph capture)
  static size_t set_sa = 0, set_ss = 0, set_sm = 0;
  if (sa > set_sa) {
    FCGNO_CUDA_TRY(cudaFuncSetAttribute(tc_analysis_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
    set_sa = sa;
  }
  if (ss > set_ss) {
    FCGNO_CUDA_TRY(cudaFuncSetAttribute(tc_synthesis_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss));
    set_ss = ss;
  }
  if (sm > set_sm) {
    FCGNO_CUDA_TRY(cudaFuncSetAttribute(tc_mix_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    set_sm = sm;
  }
  uint16_t* cur = T.va;
  uint16_t* nxt = T.vb;
  for (int l = 0; l < d.layers; ++l) {
    {
      TraceScope ts("tc_analysis", st);
      tc_analysis_kernel<C><<<dim3(g.nchunks, B), kTcThreads, sa, st>>>(g, bf16, active, cur, tab->E2, tab->G,
                                                                       T.part, d_err);
    }
    FCGNO_LAUNCHED();
    {
      TraceScope ts("tc_mix", st);
      tc_mix_kernel<C><<<dim3(g.nmodes, ceil_div(B, 128)), kTcThreads, sm, st>>>(g, B, bf16, active, T.part,
                                                                                P.Rr[l], T.chat, d_err);
    }
    FCGNO_LAUNCHED();
    SynArgs s{};
    s.g = g;
    s.B = B;
    s.bf16 = bf16;
    s.active = active;
    s.chat = T.chat;
    s.vin = cur;
    s.W = P.W[l];
    s.bias = m->w32 + BL.b[l];
    s.H = tab->H;
    s.Asyn = tab->Asyn;
    s.activate = l < d.layers - 1;
    s.vout = nxt;
    s.project = l == d.layers - 1;
    s.P1 = P.P1;
    s.p1 = m->w32 + BL.proj1_b;
    s.p2 = m->w32 + BL.proj2_w;
    s.p2b = m->w32 + BL.proj2_b;
    s.rms = rms;
    s.hh = 1.0 / ((double)(op->N + 1) * (op->N + 1));
    s.z = z;
    s.err = d_err;
    {
      TraceScope ts("tc_synthesis", st);
      tc_synthesis_kernel<C><<<dim3(g.snchunks, B), kTcThreads, ss, st>>>(s);
    }
    FCGNO_LAUNCHED();
    std::swap(cur, nxt);
  }
  return FCGNO_OK;
}

fcgno_status no_apply_tc(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms, const int* active,
                         double* z, bool fp16, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  if (!geom_supported(op->N, d.width, d.modes, d.proj_width)) {
    set_last_error("tensor-core preconditioner supports width 16 or 32 (proj_width = width), modes <= 16 and "
                   "N in {32, 64} or a multiple of 128");
    return FCGNO_EINVAL;
  }
  if (d.width == 16) return run_tc<16>(m, op, r, rms, active, z, fp16, st);
  return run_tc<32>(m, op, r, rms, active, z, fp16, st);
}

}  // namespace fcgno
