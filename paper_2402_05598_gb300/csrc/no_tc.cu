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
// The synthesis kernel's operands that do not depend on the grid point (H per column chunk,
// Asyn, W, the decoder weights and each instance's mixed coefficients) are stored as byte
// images of their shared-memory layouts, so that one bulk copy (TMA engine) stages each of
// them; the activations are stored tile-major (below), so that an activation tile is one
// contiguous bulk copy in and one out.
// Real and imaginary parts are interleaved along the contracted dimension, so every complex
// product is a real GEMM.
#include <mutex>
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
// 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))), with tanh from the hardware approximation
// (tanh.approx.f32, relative error about 2^-11): one special-function operation per value,
// so that the epilogue is not bound by the special-function unit. The tanh form departs from
// the erf form by at most 4.7e-4 and the approximate tanh adds at most 2.5e-4 |x| (absolute);
// both stay at or below the 16-bit rounding of the values produced.
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu16(float x) {
  const float u = x * fmaf(0.035677408136300125f, x * x, 0.7978845608028654f);  // sqrt(2/pi) (x + 0.044715 x^3)
  const float hx = 0.5f * x;
  return fmaf(hx, tanh_approx(u), hx);
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

// Dynamic shared memory of a synthesis block with column chunk spc and a tile ring of din
// input and dout output slots (fields of g other than SPC and KB must be set).
constexpr size_t kSynTwoPerSm = 114000;  // dynamic bytes per block that keep two blocks per SM
static size_t synthesis_bytes(const TcGeom& g, int spc, int din, int dout) {
  const size_t C = g.C, TB = 128 * C * 2, SB = (size_t)128 * g.KSYN * 2;
  const size_t SL = TB + (g.N >= 128 ? SB : 0);
  const size_t KB = (size_t)round_up(spc * 2 * g.M, 16) + 16;
  const size_t r0 = std::max((size_t)g.MP * g.KXP * 2, din * SL + dout * TB);
  return r0 + (size_t)2 * spc * g.KXP * 2 + C * KB * 2 + (g.N < 128 ? SB : 0) + 2 * C * C * 2;
}

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
  // synthesis column chunk: 32 columns when two blocks per SM still fit with a 3 + 2 slot
  // tile ring, otherwise 16. A block's set-up (the instance's mixed coefficients, stage 1 and
  // the read-back of U) does not shrink with the chunk, so wider chunks spend less of the SM's
  // copy time on it: at 64 x 64 and 256 instances a hidden layer takes 45 us with 32-column
  // chunks against 55 us with 16-column chunks (ncu, serialised launches).
  g.SPC = 16;
  if (N < 128 && g.PC >= 32 && (g.MP / 128) * 64 <= 256 && synthesis_bytes(g, 32, 3, 2) <= kSynTwoPerSm) g.SPC = 32;
  while (g.SPC % g.PT != 0) g.SPC *= 2;
  g.snchunks = N / g.SPC;
  g.KB = round_up(g.SPC * 2 * M, 16) + 16;
  g.nmodes = 2 * M * M;
  return g;
}

// 16-bit elements of an operator's activation buffers for a batch of B: each of the two
// ping-pong activation images (B n C), the partial spectral coefficients (mode x column chunk
// x block of 128 instances x 128 x 2C) and the mixed-coefficient images (B x MP x KXP).
static TcGeom narrow_geom(TcGeom g);
static void tc_acts_elems(const TcGeom& g, int B, size_t& v, size_t& part, size_t& chat) {
  const size_t nbt = ceil_div(B, 128);
  const size_t nch = std::max(g.nchunks, narrow_geom(g).nchunks);  // either launch shape
  v = (size_t)B * g.N * g.N * g.C;
  part = (size_t)g.nmodes * nch * nbt * 128 * 2 * g.C;
  chat = (size_t)B * g.MP * g.KXP;
}

static bool geom_supported(int N, int C, int M, int Cp) {
  if (!(C == 16 || C == 32) || Cp != C || M < 1 || M > 16 || N < 2 * M) return false;
  if (!(N == 32 || N == 64 || (N >= 128 && N % 128 == 0))) return false;
  if ((std::min(N, 32) * C) % 128 != 0) return false;
  // the synthesis block's two warp groups each read back whole 16-column TMEM groups of U
  if (make_geom(N, C, M).SPC % 16 != 0) return false;
  return true;
}

// ------------------------------------ tables -------------------------------------------
struct TcTables {
  int N = 0, M = 0;
  uint16_t* E2 = nullptr;    // [N / QC] images 32 x QC (K-major)
  uint16_t* G = nullptr;     // [N / PC] images NPM x 2PC (K-major)
  uint16_t* H = nullptr;     // [N / SPC] images 2SPC x KXP (K-major)
  uint16_t* Asyn = nullptr;  // images 128 x KSYN (K-major): one (N < 128) or N / 128
};

__device__ __forceinline__ void cs_of(long long k, long long x, int N, float& c, float& s) {
  const long long ph = ((k % N + N) % N) * x % N;
  double sd, cd;
  sincospi(2.0 * (double)ph / (double)N, &sd, &cd);
  c = (float)cd;
  s = (float)sd;
}

// adjoint: the tables of the transposed transforms used by the training backward: the analysis
// becomes the synthesis's adjoint (E2 rows k2 > 0 doubled, G without 1/n) and the synthesis the
// analysis's adjoint (Asyn with 1/n and without the doubling).
__global__ void tc_tables_kernel(TcGeom g, bool bf16, uint16_t* E2, uint16_t* G, uint16_t* H, uint16_t* Asyn,
                                 bool adjoint) {
  const int N = g.N, M = g.M, Ky = g.Ky;
  const float inv_n = 1.0f / ((float)N * (float)N);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  // E2: rows (k2, t) x q, one image per analysis q chunk
  if (tid < 32 * N) {
    const int row = tid / N, q = tid % N, k2 = row >> 1, t = row & 1;
    float v = 0.f;
    if (k2 < Ky) {
      float c, s;
      cs_of(k2, q, N, c, s);
      v = t ? -s : c;
      if (adjoint && k2 > 0) v *= 2.f;
    }
    E2[(size_t)(q / g.QC) * 32 * g.QC + kmajor_off(row, q % g.QC, 128, g.QC * 16) / 2] = f2h16(v, bf16);
  }
  // G: rows (j, t') x (p, t), one image per analysis column chunk
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
      if (!adjoint) v *= inv_n;
    }
    G[(size_t)(k / (2 * g.PC)) * g.NPM * 2 * g.PC + kmajor_off(row, k % (2 * g.PC), 128, 2 * g.PC * 16) / 2] =
        f2h16(v, bf16);
  }
  // H: rows (p, t') of one synthesis column chunk per image
  if (tid < 2 * N * g.KXP) {
    const int row = tid / g.KXP, k = tid % g.KXP;
    const int hc = row / (2 * g.SPC), hr = row % (2 * g.SPC);
    const int p = row >> 1, tp = row & 1, j = k >> 1, t = k & 1;
    float v = 0.f;
    if (k < g.Kx4) {
      const int k1 = j < M ? j : j - 2 * M;
      float c, s;
      cs_of(k1, p, N, c, s);
      if (tp == 0) v = t == 0 ? c : -s;
      else v = t == 0 ? s : c;
    }
    H[(size_t)hc * 2 * g.SPC * g.KXP + kmajor_off(hr, k, 128, g.KXP * 16) / 2] = f2h16(v, bf16);
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
      const float w = adjoint ? inv_n : (k2 == 0 ? 1.f : 2.f);
      v = w * (t == 0 ? c : -s);
    }
    const int img = N < 128 ? 0 : m / 128, ir = N < 128 ? m : m % 128;
    Asyn[(size_t)img * 128 * g.KSYN + kmajor_off(ir, k, 128, g.KSYN * 16) / 2] = f2h16(v, bf16);
  }
}

// ------------------------------------ model copies -------------------------------------
struct TcPrecision {
  bool built = false;
  std::vector<uint16_t*> W;   // [L] C x C image (K-major)
  std::vector<uint16_t*> Rr;  // [L] nmodes images 2C x 2C (K-major)
  std::vector<uint16_t*> WT;  // [L] images of W^T and of the transposed real mode matrices (training
  std::vector<uint16_t*> RrT; //     backward; built on demand)
  uint16_t* P1 = nullptr;     // Cp x C image (K-major)
  std::map<int, TcTables> tables;
};

}  // namespace fcgno

struct fcgno::TcModel {
  TcPrecision prec[2];  // 0: BF16, 1: FP16
};

// Training state of the BF16 path for one operator: what the backward needs from the forward
// (every layer's input and pre-activation, tile-major) and the backward's own tile-major
// gradients and partial-coefficient images. One allocation; capacities follow the op's shape.
namespace fcgno {
struct TcTrainBufs {
  size_t bytes = 0;
  void* base = nullptr;
  uint16_t* v[17] = {};       // layer inputs v_0 .. v_L (v_L: the last Fourier layer's output)
  uint16_t* h[16] = {};       // pre-activations of the layers with GELU
  uint16_t* gh = nullptr;     // gradient w.r.t. a layer's pre-activation
  uint16_t* gv = nullptr;     // gradient w.r.t. a layer's input
  uint16_t* partb = nullptr;  // partial-coefficient images of the backward's analysis
  float* gspec = nullptr;     // [B][mode][C] complex: that analysis summed over column chunks
  float* zero = nullptr;      // [C] zeros: the bias of the adjoint synthesis
  bool recompute = false;     // pre-activations rebuilt per layer in the backward (h[0] is scratch)
};
}  // namespace fcgno

struct fcgno::TcActs {
  size_t cap_v = 0, cap_part = 0, cap_chat = 0;
  uint16_t* va = nullptr;
  uint16_t* vb = nullptr;
  uint16_t* part = nullptr;  // partial-coefficient images [mode][chunk][block of 128][128 x 2C]
  uint16_t* chat = nullptr;  // mixed-coefficient images, one per instance
  int* err = nullptr;        // set to 1 by a kernel whose bounded wait ran out (kept across regrowth)
  fcgno::TcTrainBufs train;  // training (allocated on the first 16-bit training step)
};

namespace fcgno {

// rows x cols row-major FP32 -> 16-bit image of the K-major shared-memory layout (K = cols);
// transpose: the image of in^T (in is then cols x rows row-major)
__global__ void tc_cast_image_kernel(int rows, int cols, const float* __restrict__ in, uint16_t* __restrict__ out,
                                     bool bf16, bool transpose) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i / cols, k = i % cols;
  out[kmajor_off(r, k, 128, cols * 16) / 2] = f2h16(transpose ? in[k * rows + r] : in[i], bf16);
}

// Rr[mode]: image (K-major, 2C x 2C) of the real form [(o,t')][(i,t)] of R[mode][i][o][re/im];
// transpose: the image of its transpose [(i,t)][(o,t')], the real form of the conjugate
// transpose of R[mode] (the mixing's adjoint)
__global__ void tc_rr_kernel(int C, int nmodes, const float* __restrict__ R, uint16_t* __restrict__ Rr, bool bf16,
                             bool transpose) {
  const size_t total = (size_t)nmodes * 4 * C * C;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int C2 = 2 * C;
  const size_t mode = idx / (C2 * C2);
  const int rem = (int)(idx % (C2 * C2));
  const int irow = rem / C2, icol = rem % C2;
  const int row = transpose ? icol : irow, col = transpose ? irow : icol;  // element of the real form
  const int o = row >> 1, tp = row & 1, i = col >> 1, t = col & 1;
  const float re = R[((mode * C + i) * C + o) * 2], im = R[((mode * C + i) * C + o) * 2 + 1];
  float v;
  if (tp == 0) v = t == 0 ? re : -im;
  else v = t == 0 ? im : re;
  Rr[(size_t)mode * C2 * C2 + kmajor_off(irow, icol, 128, C2 * 16) / 2] = f2h16(v, bf16);
}

static void free_bwd_images(TcPrecision& p) {
  for (auto x : p.WT) cudaFree(x);
  for (auto x : p.RrT) cudaFree(x);
  p.WT.clear();
  p.RrT.clear();
}

static void free_prec(TcPrecision& p) {
  for (auto x : p.W) cudaFree(x);
  for (auto x : p.Rr) cudaFree(x);
  p.W.clear();
  p.Rr.clear();
  free_bwd_images(p);
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
  delete m->tc;
  m->tc = nullptr;
}

static void free_acts(TcActs& A) {
  uint16_t* f[] = {A.va, A.vb, A.part, A.chat};
  for (auto x : f)
    if (x) cudaFree(x);
  int* err = A.err;
  TcTrainBufs train = A.train;
  A = TcActs{};
  A.err = err;
  A.train = train;
}

void tc_acts_free(fcgno_op* op) {
  if (!op->tc_acts) return;
  if (op->tc_acts->train.base) cudaFree(op->tc_acts->train.base);
  op->tc_acts->train = TcTrainBufs{};
  free_acts(*op->tc_acts);
  if (op->tc_acts->err) cudaFree(op->tc_acts->err);
  delete op->tc_acts;
  op->tc_acts = nullptr;
}

// The operator's timeout flag, allocated (zeroed on `st`) on first use.
static fcgno_status ensure_err_flag(const fcgno_op* op, cudaStream_t st) {
  if (!op->tc_acts) op->tc_acts = new TcActs();
  TcActs& T = *op->tc_acts;
  if (T.err) return FCGNO_OK;
  if (cudaMalloc(&T.err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    T.err = nullptr;
    set_last_error("tensor-core preconditioner error flag: out of device memory");
    return FCGNO_ENOMEM;
  }
  FCGNO_CUDA_TRY(cudaMemsetAsync(T.err, 0, sizeof(int), st));
  return FCGNO_OK;
}

// Failure-detection self-test: one thread initialises an mbarrier that expects one arrival,
// which nothing provides, and waits for its first phase through the bounded wait of the
// tensor-core kernels with the given limit. When the wait gives up it raises the timeout
// flag exactly as those kernels do. Nothing is in flight: no copy, MMA or TMEM allocation.
__global__ void wait_probe_kernel(uint64_t limit_ns, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  if (!mbar_wait(&bar, 0, limit_ns)) atomicExch(err, 1);
}

fcgno_status tc_wait_probe(const fcgno_op* op, uint64_t limit_ns, cudaStream_t st) {
  FCGNO_TRY(ensure_err_flag(op, st));
  wait_probe_kernel<<<1, 32, 0, st>>>(limit_ns, op->tc_acts->err);
  FCGNO_LAUNCHED();
  return tc_take_timeout(op, st);
}

fcgno_status tc_take_timeout(const fcgno_op* op, cudaStream_t st) {
  if (!op->tc_acts || !op->tc_acts->err) return FCGNO_OK;
  int flag = 0;
  FCGNO_CUDA_TRY(cudaMemcpyAsync(&flag, op->tc_acts->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  FCGNO_CUDA_TRY(cudaStreamSynchronize(st));
  if (flag == 0) return FCGNO_OK;
  FCGNO_CUDA_TRY(cudaMemsetAsync(op->tc_acts->err, 0, sizeof(int), st));
  set_last_error("a tensor-core preconditioner kernel gave up a bounded device wait: "
                 "preconditioner outputs on this operator since the last check are invalid");
  return FCGNO_ETIMEOUT;
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
      free_bwd_images(p);
      if (p.P1) cudaFree(p.P1);
      p.P1 = nullptr;
      p.built = false;
    }
  return FCGNO_OK;
}

// The 16-bit weight images of the forward (W, Rr per layer and the decoder's first layer),
// cast from the FP32 master blob into their existing buffers.
static fcgno_status cast_images(fcgno_model* m, TcPrecision& P, bool bf16, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  const int C = d.width, Cp = d.proj_width, nmodes = 2 * d.modes * d.modes;
  BlobLayout BL = blob_layout(d);
  const size_t tot = (size_t)nmodes * 4 * C * C;
  for (int l = 0; l < d.layers; ++l) {
    tc_cast_image_kernel<<<ceil_div(C * C, 256), 256, 0, st>>>(C, C, m->w32 + BL.w[l], P.W[l], bf16, false);
    FCGNO_LAUNCHED();
    tc_rr_kernel<<<ceil_div(tot, 256), 256, 0, st>>>(C, nmodes, m->w32 + BL.r[l], P.Rr[l], bf16, false);
    FCGNO_LAUNCHED();
  }
  tc_cast_image_kernel<<<ceil_div(Cp * C, 256), 256, 0, st>>>(Cp, C, m->w32 + BL.proj1_w, P.P1, bf16, false);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

static fcgno_status ensure_prec(fcgno_model* m, bool fp16, cudaStream_t st) {
  if (!m->tc) m->tc = new TcModel();
  TcPrecision& P = m->tc->prec[fp16 ? 1 : 0];
  if (P.built) return FCGNO_OK;
  const fcgno_model_desc& d = m->desc;
  const int C = d.width, Cp = d.proj_width, M = d.modes, nmodes = 2 * M * M;
  P.W.assign(d.layers, nullptr);
  P.Rr.assign(d.layers, nullptr);
  for (int l = 0; l < d.layers; ++l) {
    FCGNO_CUDA_TRY(cudaMalloc(&P.W[l], sizeof(uint16_t) * C * C));
    FCGNO_CUDA_TRY(cudaMalloc(&P.Rr[l], sizeof(uint16_t) * (size_t)nmodes * 4 * C * C));
  }
  FCGNO_CUDA_TRY(cudaMalloc(&P.P1, sizeof(uint16_t) * Cp * C));
  FCGNO_TRY(cast_images(m, P, !fp16, st));
  P.built = true;
  m->gen++;
  return FCGNO_OK;
}

static fcgno_status ensure_tables(fcgno_model* m, bool fp16, const TcGeom& g, TcTables*& out, cudaStream_t st,
                                  bool adjoint = false) {
  TcPrecision& P = m->tc->prec[fp16 ? 1 : 0];
  // the analysis tables depend on the column-chunk width; adjoint tables serve the training backward
  const int key = (g.N * 256 + g.PC) * 2 + (adjoint ? 1 : 0);
  auto it = P.tables.find(key);
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
  tc_tables_kernel<<<ceil_div(work, 256), 256, 0, st>>>(g, !fp16, t.E2, t.G, t.H, t.Asyn, adjoint);
  FCGNO_LAUNCHED();
  P.tables[key] = t;
  out = &P.tables[key];
  m->gen++;
  return FCGNO_OK;
}

// ------------------------------------ kernels ------------------------------------------
__device__ __forceinline__ bool tc_inactive(const int* active, int b) { return active && active[b] >= 0; }

// Tile-major activation layout (16-bit). An instance's N x N x C activations are N^2/128
// tiles of 128 grid points, stored one after another; each tile is the byte image of a
// K-major tensor-core operand (rows = grid points, K = channels; LBO 2048, SBO 128):
//   N < 128 : tile tau holds the PT = 128/N grid columns tau*PT .. tau*PT + PT - 1, all rows;
//   N >= 128: tile tau holds column tau % N, rows 128 (tau / N) .. + 127.
// Row m of a tile = (column within the tile) * QT + (row within the tile); element (m, c) is
// at byte (c / 8) * 2048 + m * 16 + (c % 8) * 2. The same bytes, read with the 8-channel
// groups as the M direction, are the MN-major operand of the analysis stage Q (K = rows q).
__host__ __device__ __forceinline__ void act_tile_of(const TcGeom& g, int q, int p, int& tile, int& m) {
  if (g.N < 128) {
    tile = p / g.PT;
    m = (p % g.PT) * g.N + q;
  } else {
    tile = (q / 128) * g.N + p;
    m = q % 128;
  }
}

// Encoder: v0 = lift_w [r/rms, log k] + lift_b, written tile-major. One block covers
// kLiftCols grid columns of kLiftRows(N) = min(N, 128) rows of one instance, i.e. whole tiles:
// it reads those rows of r (FP64) and log k (FP32) with coalesced row segments into shared
// memory, then writes the tiles' 16-byte channel-group rows in order, consecutive threads on
// consecutive tile rows. 1/rms is formed once per thread in FP32.
constexpr int kLiftCols = 32, kLiftThreads = 256;
__host__ __device__ constexpr int lift_rows(int N) { return N < 128 ? N : 128; }
template <int C>
__global__ void __launch_bounds__(kLiftThreads) tc_lift_kernel(TcGeom g, const double* __restrict__ r,
                                                               const float* __restrict__ logk,
                                                               const double* __restrict__ rms,
                                                               const int* __restrict__ active,
                                                               const float* __restrict__ lw,
                                                               const float* __restrict__ lb,
                                                               uint16_t* __restrict__ v, bool bf16) {
  __shared__ float w0[C], w1[C], bb[C];
  __shared__ float2 sv[128][kLiftCols + 1];  // (r / rms, log k) of the block's grid points
  pdl_wait();  // r, rms and the status flags come from the FCG step just before
  pdl_trigger();
  const int b = blockIdx.y;
  if (tc_inactive(active, b)) return;
  const int tid = threadIdx.x;
  for (int c = tid; c < C; c += kLiftThreads) {
    w0[c] = lw[2 * c];
    w1[c] = lw[2 * c + 1];
    bb[c] = lb[c];
  }
  const int N = g.N, R = lift_rows(N), ncol = N / kLiftCols;
  const int p0 = (blockIdx.x % ncol) * kLiftCols, q0 = (blockIdx.x / ncol) * R;
  const size_t n = (size_t)N * N;
  const float s = (float)rms[b];
  const float inv = s > 0.f ? 1.0f / s : 0.f;
  const double* rb = r + (size_t)b * n;
  const float* lb_ = logk + (size_t)b * n;
  // every load of the thread is issued before the first shared-memory store
  constexpr int kLoads = 128 * kLiftCols / kLiftThreads;
  double rv[kLoads];
  float lv[kLoads];
#pragma unroll
  for (int i = 0; i < kLoads; ++i) {
    const int idx = tid + i * kLiftThreads, qq = idx / kLiftCols, pp = idx % kLiftCols;
    if (idx < R * kLiftCols) {
      const size_t pt = (size_t)(q0 + qq) * N + p0 + pp;
      rv[i] = rb[pt];
      lv[i] = lb_[pt];
    }
  }
#pragma unroll
  for (int i = 0; i < kLoads; ++i) {
    const int idx = tid + i * kLiftThreads;
    if (idx < R * kLiftCols) sv[idx / kLiftCols][idx % kLiftCols] = make_float2((float)rv[i] * inv, lv[i]);
  }
  __syncthreads();
  // tiles of the block: N < 128: PT columns x N rows each; N >= 128: one column x 128 rows
  const int ntl = R * kLiftCols / 128;
  const size_t tau0 = N < 128 ? (size_t)(p0 / g.PT) : (size_t)(q0 / 128) * N + p0;
  constexpr int CG = C / 8;
  for (int idx = tid; idx < ntl * CG * 128; idx += kLiftThreads) {
    const int m = idx % 128, cg = (idx / 128) % CG, tl = idx / (128 * CG);
    int row, col;
    if (N < 128) {
      col = tl * g.PT + m / N;
      row = m % N;
    } else {
      col = tl;
      row = m;
    }
    const float2 x = sv[row][col];
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = cg * 8 + 2 * i;
      w[i] = pack2(fmaf(w0[c], x.x, fmaf(w1[c], x.y, bb[c])), fmaf(w0[c + 1], x.x, fmaf(w1[c + 1], x.y, bb[c + 1])),
                   bf16);
    }
    uint8_t* dst = reinterpret_cast<uint8_t*>(v + ((size_t)b * n + (tau0 + tl) * 128) * C) + cg * 2048 + m * 16;
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Truncated analysis of one grid-column chunk of one instance; writes its 16-bit partial
// coefficients into the mode-mixing operand images (see tc_mix_kernel).
//
// Stage Q runs over steps s = (m-tile, q chunk); an m-tile is 128/C grid columns x C channels
// (M) and a q chunk QC rows (K). Its operand is copied straight from the tile-major
// activations: for N < 128 one bulk copy of (128/C)/PT consecutive tiles, for N >= 128 one
// copy of QC rows per (column, 8-channel group). M groups of 8 channels are ordered
// (tile u, channel group cg, column within the tile pl) and sit QC*16 bytes apart.
// Warp-specialised: warps 0-3 read the Z accumulators back and store the result; lane 0 of
// warp 4 issues the MMAs and lane 0 of warp 5 the bulk copies, through a three-slot ring; the
// roles meet only on mbarriers. Z accumulators rotate through up to eight 32-column TMEM
// slots, which overlap the stage-P accumulators (stage P starts only after every Z has been
// read back), so that the MMAs are not held back by the read-back.
constexpr int kAnaThreads = 192;
template <int C>
__global__ void __launch_bounds__(kAnaThreads, 2)
    tc_analysis_kernel(TcGeom g, int nbt, bool bf16, const int* __restrict__ active, const uint16_t* __restrict__ v,
                       const uint16_t* __restrict__ E2, const uint16_t* __restrict__ G, uint16_t* __restrict__ part,
                       int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int NS = 3;
  // full[s] step copied in; sfree[s] its MMAs done; zfull[z] / zempty[z] Z slot ready / read
  // back (4 warp arrivals); prob prologue copies; apready stage-P operand complete (4); pfull
  // stage-P accumulators ready
  constexpr int NZ = 8;
  __shared__ uint64_t full[NS], sfree[NS], zfull[NZ], zempty[NZ], prob, apready, pfull;
  __shared__ uint32_t tbase_s;
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (tc_inactive(active, b)) return;
  const int N = g.N, PC = g.PC, QC = g.QC, Ky = g.Ky, PT = g.PT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int qchunks = N / QC;
  const int ne2 = qchunks > 1 ? NS : 1;  // E2 changes per q chunk only when N > QC
  const uint32_t E2B = 32 * QC * 2, AB = 128 * QC * 2, GB = g.NPM * 2 * PC * 2;
  uint8_t* sE2 = smem;                            // ne2 x (32 x QC), K-major: LBO 128, SBO QC*16
  uint8_t* sA = sE2 + ne2 * E2B;                  // NS x (128 x QC), MN-major: LBO 128, SBO QC*16
  uint8_t* sAP = sA + NS * AB;                    // MP x 2PC, K-major: LBO 128, SBO 2PC*16
  uint8_t* sG = sAP + (size_t)g.MP * 2 * PC * 2;  // NPM x 2PC, K-major: LBO 128, SBO 2PC*16
  const uint32_t SBO_E = QC * 16, SBO_A = QC * 16, SBO_P = 2 * PC * 16, SBO_G = 2 * PC * 16;
  const uint32_t tcols = ((g.MP / 128) * g.NPM) <= 256 ? 256u : 512u;
  if (warp == 0) tmem_alloc(&tbase_s, tcols);
  if (tid == 128) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&sfree[i], 1);
    }
    for (int i = 0; i < NZ; ++i) {
      mbar_init(&zfull[i], 1);
      mbar_init(&zempty[i], 4);
    }
    mbar_init(&prob, 1);
    mbar_init(&apready, 4);
    mbar_init(&pfull, 1);
  }
  // zero the padding rows of sAP
  for (int idx = tid; idx < (g.MP - Ky * C) * (2 * PC / 8); idx += kAnaThreads) {
    const int row = Ky * C + idx / (2 * PC / 8), kc = idx % (2 * PC / 8);
    *reinterpret_cast<uint4*>(sAP + kmajor_off(row, kc * 8, 128, SBO_P)) = make_uint4(0, 0, 0, 0);
  }
  fence_smem_to_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tbase_s;
  const uint32_t tP = tbase;  // stage-P accumulators (after stage Q)
  const uint32_t tQ = tbase;  // nz Z slots of 32 columns (stage Q)
  const int nz = (int)(tcols / 32) < NZ ? (int)(tcols / 32) : NZ;
  const int p0 = chunk * PC;
  const int cols_mt = 128 / C;  // grid columns per m-tile
  const int mtiles = PC / cols_mt;
  const int nsteps = mtiles * qchunks;
  const int ptiles = g.MP / 128;
  bool ok = true;
  if (warp == 4) {
    // ================================ MMA issuer (one lane) ============================
    if (lane == 0) {
      int mmas = 0;
      bool p_pending = false;
      const uint32_t idQ = idesc_f16(128, 32, bf16, true, false);
      ok = mbar_wait(&prob, 0);
      for (int s = 0; s < nsteps && ok; ++s) {
        const int buf = s % NS, mt = s / qchunks, qc = s % qchunks;
        ok = mbar_wait(&full[buf], (s / NS) & 1);
        if (ok && qc == 0 && mt >= nz) ok = mbar_wait(&zempty[mt % nz], ((mt / nz) - 1) & 1);
        if (!ok) break;
        fence_after_sync();
        const uint32_t tq = tQ + (mt % nz) * 32;
        const uint32_t sa = smem_addr(sA + buf * AB);
        const uint32_t e2 = smem_addr(sE2 + (qchunks > 1 ? buf * E2B : 0));
        for (int ks = 0; ks < QC / 16; ++ks)
          mma(tq, desc(sa + ks * 256, 128, SBO_A), desc(e2 + ks * 256, 128, SBO_E), idQ, qc > 0 || ks > 0);
        commit(&sfree[buf]);
        if (qc == qchunks - 1) commit(&zfull[mt % nz]);
        mmas = s + 1;
      }
      if (ok) ok = mbar_wait(&apready, 0);  // every Z read back into sAP
      if (ok) {
        fence_after_sync();
        const uint32_t id = idesc_f16(128, g.NPM, bf16, false, false);
        for (int pt = 0; pt < ptiles; ++pt)
          for (int ks = 0; ks < 2 * PC / 16; ++ks) {
            const uint64_t ad = desc(smem_addr(sAP) + pt * 16 * SBO_P + ks * 2 * 128, 128, SBO_P);
            const uint64_t bd = desc(smem_addr(sG) + ks * 2 * 128, 128, SBO_G);
            mma(tP + pt * g.NPM, ad, bd, id, ks > 0);
          }
        commit(&pfull);
        p_pending = true;
      }
      if (!ok) {
        // error path: let the MMAs this block started finish (bounded)
        for (int u = mmas > NS ? mmas - NS : 0; u < mmas; ++u) mbar_wait(&sfree[u % NS], (u / NS) & 1);
        atomicExch(err, 1);
      }
      if (p_pending) mbar_wait(&pfull, 0);  // (the read-back warps wait on it too)
    }
  } else if (warp == 5) {
    // ================================ load issuer (one lane) ===========================
    if (lane == 0) {
      const uint16_t* vb = v + (size_t)b * N * N * C;
      int loads = 0;
      auto stage = [&](int s) {
        const int buf = s % NS, mt = s / qchunks, qc = s % qchunks;
        const int pm = p0 + mt * cols_mt;  // first grid column of the m-tile
        mbar_expect_tx(&full[buf], AB + (qchunks > 1 ? E2B : 0));
        if (qchunks > 1) bulk_g2s(sE2 + buf * E2B, E2 + (size_t)qc * 32 * QC, E2B, &full[buf]);
        uint8_t* dst = sA + buf * AB;
        if (N < 128) {
          bulk_g2s(dst, vb + (size_t)(pm / PT) * 128 * C, AB, &full[buf]);
        } else {
          const int q0 = qc * QC, qt = q0 / 128, ql = q0 % 128;
          for (int u = 0; u < cols_mt; ++u)
            for (int cg = 0; cg < C / 8; ++cg)
              bulk_g2s(dst + (u * (C / 8) + cg) * QC * 16,
                       vb + (size_t)(qt * N + pm + u) * 128 * C + cg * 1024 + ql * 8, QC * 16, &full[buf]);
        }
        loads = s + 1;
      };
      mbar_expect_tx(&prob, GB + (qchunks == 1 ? E2B : 0));
      bulk_g2s(sG, G + (size_t)chunk * g.NPM * 2 * PC, GB, &prob);
      if (qchunks == 1) bulk_g2s(sE2, E2, E2B, &prob);
      pdl_wait();  // the activations come from the kernel just before
      pdl_trigger();
      for (int s = 0; s < nsteps && ok; ++s) {
        if (s >= NS) ok = mbar_wait(&sfree[s % NS], ((s / NS) - 1) & 1);  // step s-NS's MMAs read the slot
        if (ok) stage(s);
      }
      if (!ok) {
        for (int u = loads > NS ? loads - NS : 0; u < loads; ++u) mbar_wait(&full[u % NS], (u / NS) & 1);
        atomicExch(err, 1);
      }
      mbar_wait(&prob, 0);
    }
  } else {
    // ================================ read-back warps 0-3 ==============================
    // Z of m-tile mt: lane M -> (column, channel), columns (k2, t) -> sAP[(k2, c)][(p, t)]
    pdl_wait();  // (before their global writes)
    const int M = warp * 32 + lane, Gi = M >> 3;
    const int u = Gi / ((C / 8) * PT), cg = (Gi / PT) % (C / 8), pl2 = Gi % PT;
    const int c = cg * 8 + (M & 7);
    for (int mt = 0; mt < mtiles && ok; ++mt) {
      ok = mbar_wait(&zfull[mt % nz], (mt / nz) & 1);
      if (!ok) break;
      fence_after_sync();
      const uint32_t tq = tQ + (mt % nz) * 32 + ((uint32_t)(warp * 32) << 16);
      float z[32];
      float tmp[16];
      tmem_ld16(tq, tmp);
#pragma unroll
      for (int i = 0; i < 16; ++i) z[i] = tmp[i];
      tmem_ld16(tq + 16, tmp);
#pragma unroll
      for (int i = 0; i < 16; ++i) z[16 + i] = tmp[i];
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&zempty[mt % nz]);
      const int pl = mt * cols_mt + u * PT + pl2;
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {  // Ky <= 16: static indices keep z in registers
        if (k2 < Ky) {
          const int row = k2 * C + c;
          *reinterpret_cast<uint32_t*>(sAP + kmajor_off(row, 2 * pl, 128, SBO_P)) =
              pack2(z[2 * k2], z[2 * k2 + 1], bf16);
        }
      }
    }
    if (ok) {
      fence_smem_to_async();
      fence_before_sync();  // every Z read of this warp precedes stage P (same TMEM columns)
      __syncwarp();
      if (lane == 0) mbar_arrive(&apready);
      ok = mbar_wait(&pfull, 0);
      fence_after_sync();
    }
    if (ok) {
      // P row (k2, c), columns (j, t') -> image of mode j*Ky + k2, row b % 128, K (c, t')
      const size_t img = (size_t)128 * 2 * C;  // elements per image
      const int bt = b / 128, br = b % 128;
      for (int pt = 0; pt < ptiles; ++pt) {
        const int row = pt * 128 + warp * 32 + lane;
        const int k2 = row / C, cc = row % C;
        const uint32_t off = kmajor_off(br, 2 * cc, 128, 2 * C * 16) / 2;
        for (int c0 = 0; c0 < g.NPM; c0 += 16) {
          float val[16];
          tmem_ld16(tP + pt * g.NPM + c0 + ((uint32_t)(warp * 32) << 16), val);
          if (row < Ky * C) {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
              const int j = (c0 + i) >> 1;
              if (j < 2 * g.M) {
                const int mode = j * Ky + k2;
                uint16_t* dst = part + (((size_t)mode * g.nchunks + chunk) * nbt + bt) * img + off;
                *reinterpret_cast<uint32_t*>(dst) = pack2(val[i], val[i + 1], bf16);
              }
            }
          }
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, tcols);
}

// Persistent form of tc_analysis_kernel for the wide launch shape at N < 128 (one q chunk):
// each block keeps one column chunk and walks the active instances b0, b0 + stride, ... of it,
// so that one item's stage P, read-back and stores overlap the next item's copies and stage-Q
// MMAs. Roles: warps 0-3 read the Z accumulators back into the stage-P operand, lane 0 of
// warp 4 issues the MMAs, lane 0 of warp 5 the bulk copies (ring of NS slots, continuing across
// items), warps 6-9 read stage P back and store the partial coefficients. TMEM: the stage-P
// accumulators in the first ptiles x NPM columns, NZ Z slots of 32 columns in the last ones
// (disjoint, so the next item's stage Q runs while stage P is read back). Hand-offs per item:
// apready (every Z of the item staged), pfull (stage P done: its accumulators readable, the
// stage-P operand free again), pempty (stage P read back: its accumulators free again).
constexpr int kAnaPipeThreads = 320, kAnaPipeZ = 3;
template <int C>
__global__ void __launch_bounds__(kAnaPipeThreads, 2)
    tc_analysis_pipe_kernel(TcGeom g, int B, int nbt, bool bf16, const int* __restrict__ active,
                            const uint16_t* __restrict__ v, const uint16_t* __restrict__ E2,
                            const uint16_t* __restrict__ G, uint16_t* __restrict__ part, int* __restrict__ err,
                            int rev) {
  // rev: walk the instances from the last to the first. The layer input was written in
  // increasing instance order, so its last instances are the likeliest to be still in L2.
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int NS = 3, NZ = kAnaPipeZ;
  __shared__ uint64_t full[NS], sfree[NS], zfull[NZ], zempty[NZ], prob, apready, pfull, pempty;
  __shared__ uint32_t tbase_s;
  const int N = g.N, PC = g.PC, QC = g.QC, Ky = g.Ky, PT = g.PT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t E2B = 32 * QC * 2, AB = 128 * QC * 2, GB = g.NPM * 2 * PC * 2;
  uint8_t* sE2 = smem;                            // 32 x QC, K-major: LBO 128, SBO QC*16
  uint8_t* sA = sE2 + E2B;                        // NS x (128 x QC), MN-major: LBO 128, SBO QC*16
  uint8_t* sAP = sA + NS * AB;                    // MP x 2PC, K-major: LBO 128, SBO 2PC*16
  uint8_t* sG = sAP + (size_t)g.MP * 2 * PC * 2;  // NPM x 2PC, K-major: LBO 128, SBO 2PC*16
  const uint32_t SBO_E = QC * 16, SBO_A = QC * 16, SBO_P = 2 * PC * 16, SBO_G = 2 * PC * 16;
  constexpr uint32_t tcols = 256;
  const int chunk = blockIdx.x % g.nchunks;
  const int b0 = blockIdx.x / g.nchunks, bstride = gridDim.x / g.nchunks;
  if (warp == 0) tmem_alloc(&tbase_s, tcols);
  if (tid == 128) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&sfree[i], 1);
    }
    for (int i = 0; i < NZ; ++i) {
      mbar_init(&zfull[i], 1);
      mbar_init(&zempty[i], 4);
    }
    mbar_init(&prob, 1);
    mbar_init(&apready, 4);
    mbar_init(&pfull, 1);
    mbar_init(&pempty, 4);
  }
  // zero the padding rows of sAP (never written by the Z read-back)
  for (int idx = tid; idx < (g.MP - Ky * C) * (2 * PC / 8); idx += kAnaPipeThreads) {
    const int row = Ky * C + idx / (2 * PC / 8), kc = idx % (2 * PC / 8);
    *reinterpret_cast<uint4*>(sAP + kmajor_off(row, kc * 8, 128, SBO_P)) = make_uint4(0, 0, 0, 0);
  }
  fence_smem_to_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tbase_s;
  const uint32_t tP = tbase;                        // ptiles x NPM stage-P columns
  const uint32_t tQ = tbase + tcols - NZ * 32;      // NZ Z slots
  const int p0 = chunk * PC;
  const int cols_mt = 128 / C;                      // grid columns per m-tile
  const int mtiles = PC / cols_mt;
  const int ptiles = g.MP / 128;
  bool ok = true;
  // Every role skips the stopped instances on its own, and the MMA issuer and the Z read-back
  // read the status flags without waiting on the programmatic link. They all see the same flags
  // because this kernel never directly follows the FCG step that sets them: the encoder or a
  // synthesis runs in between, and those trigger their successor only after their own wait.
  if (warp == 4) {
    // ================================ MMA issuer (one lane) ============================
    if (lane == 0) {
      int gstep = 0, mmas = 0, item = 0, pissued = 0;
      const uint32_t idQ = idesc_f16(128, 32, bf16, true, false);
      const uint32_t idP = idesc_f16(128, g.NPM, bf16, false, false);
      ok = mbar_wait(&prob, 0);
      for (int bb = b0; bb < B && ok; bb += bstride) {
        const int b = rev ? B - 1 - bb : bb;
        if (tc_inactive(active, b)) continue;
        for (int mt = 0; mt < mtiles && ok; ++mt, ++gstep) {
          const int buf = gstep % NS;
          ok = mbar_wait(&full[buf], (gstep / NS) & 1);
          if (ok && gstep >= NZ) ok = mbar_wait(&zempty[gstep % NZ], ((gstep / NZ) - 1) & 1);
          if (!ok) break;
          fence_after_sync();
          const uint32_t tq = tQ + (gstep % NZ) * 32;
          const uint32_t sa = smem_addr(sA + buf * AB), e2 = smem_addr(sE2);
          for (int ks = 0; ks < QC / 16; ++ks)
            mma(tq, desc(sa + ks * 256, 128, SBO_A), desc(e2 + ks * 256, 128, SBO_E), idQ, ks > 0);
          commit(&sfree[buf]);
          commit(&zfull[gstep % NZ]);
          mmas = gstep + 1;
        }
        if (ok) ok = mbar_wait(&apready, item & 1);                       // every Z of the item staged
        if (ok && item > 0) ok = mbar_wait(&pempty, (item - 1) & 1);      // previous stage P read back
        if (ok) {
          fence_after_sync();
          for (int pt = 0; pt < ptiles; ++pt)
            for (int ks = 0; ks < 2 * PC / 16; ++ks) {
              const uint64_t ad = desc(smem_addr(sAP) + pt * 16 * SBO_P + ks * 2 * 128, 128, SBO_P);
              const uint64_t bd = desc(smem_addr(sG) + ks * 2 * 128, 128, SBO_G);
              mma(tP + pt * g.NPM, ad, bd, idP, ks > 0);
            }
          commit(&pfull);
          pissued = item + 1;
        }
        ++item;
      }
      if (!ok) {
        // error path: let the MMAs this block started finish (bounded)
        for (int u = mmas > NS ? mmas - NS : 0; u < mmas; ++u) mbar_wait(&sfree[u % NS], (u / NS) & 1);
        if (pissued > 0) mbar_wait(&pfull, (pissued - 1) & 1);
        atomicExch(err, 1);
      }
    }
  } else if (warp == 5) {
    // ================================ load issuer (one lane) ===========================
    if (lane == 0) {
      int gstep = 0, loads = 0;
      mbar_expect_tx(&prob, GB + E2B);
      bulk_g2s(sG, G + (size_t)chunk * g.NPM * 2 * PC, GB, &prob);
      bulk_g2s(sE2, E2, E2B, &prob);
      pdl_wait();  // the activations come from the kernel just before
      pdl_trigger();
      for (int bb = b0; bb < B && ok; bb += bstride) {
        const int b = rev ? B - 1 - bb : bb;
        if (tc_inactive(active, b)) continue;
        const uint16_t* vb = v + (size_t)b * N * N * C;
        for (int mt = 0; mt < mtiles && ok; ++mt, ++gstep) {
          if (gstep >= NS) ok = mbar_wait(&sfree[gstep % NS], ((gstep / NS) - 1) & 1);  // slot read
          if (!ok) break;
          const int buf = gstep % NS, pm = p0 + mt * cols_mt;
          mbar_expect_tx(&full[buf], AB);
          bulk_g2s(sA + buf * AB, vb + (size_t)(pm / PT) * 128 * C, AB, &full[buf]);
          loads = gstep + 1;
        }
      }
      if (!ok) {
        for (int u = loads > NS ? loads - NS : 0; u < loads; ++u) mbar_wait(&full[u % NS], (u / NS) & 1);
        atomicExch(err, 1);
      }
      mbar_wait(&prob, 0);
    }
  } else if (warp < 4) {
    // ================================ Z read-back warps 0-3 ============================
    // Z of an m-tile: lane M -> (column, channel), columns (k2, t) -> sAP[(k2, c)][(p, t)]
    const int M = warp * 32 + lane, Gi = M >> 3;
    const int u = Gi / ((C / 8) * PT), cg = (Gi / PT) % (C / 8), pl2 = Gi % PT;
    const int c = cg * 8 + (M & 7);
    int gmt = 0, item = 0;
    for (int bb = b0; bb < B && ok; bb += bstride) {
        const int b = rev ? B - 1 - bb : bb;
      if (tc_inactive(active, b)) continue;
      if (item > 0) {
        ok = mbar_wait(&pfull, (item - 1) & 1);  // the previous item's stage P has read sAP
        fence_after_sync();
      }
      for (int mt = 0; mt < mtiles && ok; ++mt, ++gmt) {
        ok = mbar_wait(&zfull[gmt % NZ], (gmt / NZ) & 1);
        if (!ok) break;
        fence_after_sync();
        const uint32_t tq = tQ + (gmt % NZ) * 32 + ((uint32_t)(warp * 32) << 16);
        float z[32];
        float tmp[16];
        tmem_ld16(tq, tmp);
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = tmp[i];
        tmem_ld16(tq + 16, tmp);
#pragma unroll
        for (int i = 0; i < 16; ++i) z[16 + i] = tmp[i];
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&zempty[gmt % NZ]);
        const int pl = mt * cols_mt + u * PT + pl2;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {  // Ky <= 16: static indices keep z in registers
          if (k2 < Ky) {
            const int row = k2 * C + c;
            *reinterpret_cast<uint32_t*>(sAP + kmajor_off(row, 2 * pl, 128, SBO_P)) =
                pack2(z[2 * k2], z[2 * k2 + 1], bf16);
          }
        }
      }
      if (!ok) break;
      fence_smem_to_async();
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&apready);
      ++item;
    }
  } else {
    // ================================ stage-P read-back warps 6-9 ======================
    pdl_wait();  // (before their global writes)
    const int q = warp & 3;  // TMEM lane quadrant of this warp
    const size_t img = (size_t)128 * 2 * C;  // elements per image
    int item = 0;
    for (int bb = b0; bb < B && ok; bb += bstride) {
        const int b = rev ? B - 1 - bb : bb;
      if (tc_inactive(active, b)) continue;
      ok = mbar_wait(&pfull, item & 1);
      if (!ok) break;
      fence_after_sync();
      // P row (k2, c), columns (j, t') -> image of mode j*Ky + k2, row b % 128, K (c, t')
      const int bt = b / 128, br = b % 128;
      for (int pt = 0; pt < ptiles; ++pt) {
        const int row = pt * 128 + q * 32 + lane;
        const int k2 = row / C, cc = row % C;
        const uint32_t off = kmajor_off(br, 2 * cc, 128, 2 * C * 16) / 2;
        for (int c0 = 0; c0 < g.NPM; c0 += 16) {
          float val[16];
          tmem_ld16(tP + pt * g.NPM + c0 + ((uint32_t)(q * 32) << 16), val);
          if (row < Ky * C) {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
              const int j = (c0 + i) >> 1;
              if (j < 2 * g.M) {
                const int mode = j * Ky + k2;
                uint16_t* dst = part + (((size_t)mode * g.nchunks + chunk) * nbt + bt) * img + off;
                *reinterpret_cast<uint32_t*>(dst) = pack2(val[i], val[i + 1], bf16);
              }
            }
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&pempty);
      ++item;
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, tcols);
}

// Whether the persistent analysis applies to geometry g: one q chunk (N < 128) and the stage-P
// accumulators beside the Z slots in a block's 256 TMEM columns.
static bool ana_pipe_ok(const TcGeom& g) {
  return g.N < 128 && g.N / g.QC == 1 && (g.MP / 128) * g.NPM + kAnaPipeZ * 32 <= 256;
}

// Blocks of the persistent analysis: two per SM (a multiple of the column chunks), at most one
// per (chunk, instance).
static int ana_pipe_blocks(const TcGeom& g, int B) {
  // the SM count, read once (a function-local static: initialised once even with concurrent callers)
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  const int per = std::max(1, (2 * sms) / g.nchunks);
  return g.nchunks * std::min(per, B);
}

// Per-mode complex channel mixing across instances: rows = instances (128 per CTA).
// Input: for each column chunk the 16-bit partial-coefficient image of this (mode, block of
// 128 instances), 128 x 2C K-major (K = (c, re/im)); the MMA sums the chunks in its FP32
// accumulator. Output: for each instance the byte image (MP x KXP, 16-bit, zero padded) of
// the synthesis stage-1 A operand in its MN-major shared-memory layout, element
// (m = (k2, c), k = (j, re/im)); each instance's 8 consecutive outputs c of one
// (mode, re/im) form one 16-byte run.
constexpr int kMixSlots = 4;
template <int C>
__global__ void __launch_bounds__(kTcThreads, 4)
    tc_mix_kernel(TcGeom g, int B, int nbt, bool bf16, const int* __restrict__ active,
                  const uint16_t* __restrict__ part, const uint16_t* __restrict__ Rr, uint16_t* __restrict__ chat,
                  int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t full[kMixSlots], sfree[kMixSlots], rbar, accb;
  __shared__ uint32_t tbase_s;
  __shared__ int any_active;
  constexpr int C2 = 2 * C;
  constexpr uint32_t AB = 128 * C2 * 2, RB = C2 * C2 * 2, SBO = C2 * 16;
  constexpr uint32_t TCOLS = C2 < 32 ? 32 : C2;
  const int mode = blockIdx.x, bt = blockIdx.y, b0 = bt * 128;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) any_active = 0;
  __syncthreads();
  if (b0 + tid < B && !tc_inactive(active, b0 + tid)) any_active = 1;
  __syncthreads();
  if (!any_active) return;  // every instance of this tile has stopped
  const int nch = g.nchunks, MS = nch < kMixSlots ? nch : kMixSlots;
  uint8_t* sR = smem;       // C2 x C2 image, K-major
  uint8_t* sA = smem + RB;  // MS slots of 128 x C2 images, K-major
  if (warp == 0) tmem_alloc(&tbase_s, TCOLS);
  if (tid == 0) {
    for (int i = 0; i < MS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&sfree[i], 1);
    }
    mbar_init(&rbar, 1);
    mbar_init(&accb, 1);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tbase_s;
  bool ok = true;
  if (tid != 0) pdl_wait();  // (before the read-back's global writes)
  if (tid == 0) {
    const uint16_t* pm = part + (size_t)mode * nch * nbt * 128 * C2;
    auto load = [&](int ch) {
      mbar_expect_tx(&full[ch % MS], AB);
      bulk_g2s(sA + (ch % MS) * AB, pm + ((size_t)ch * nbt + bt) * 128 * C2, AB, &full[ch % MS]);
    };
    mbar_expect_tx(&rbar, RB);
    bulk_g2s(sR, Rr + (size_t)mode * C2 * C2, RB, &rbar);
    pdl_wait();  // the partial coefficients come from the analysis just before
    pdl_trigger();
    for (int ch = 0; ch < MS; ++ch) load(ch);
    ok = mbar_wait(&rbar, 0);
    const uint32_t id = idesc_f16(128, C2, bf16, false, false);
    int issued = MS, mmas = 0;
    for (int ch = 0; ch < nch && ok; ++ch) {
      ok = mbar_wait(&full[ch % MS], (ch / MS) & 1);
      if (!ok) break;
      const uint32_t sa = smem_addr(sA + (ch % MS) * AB);
      for (int ks = 0; ks < C2 / 16; ++ks)
        mma(tbase, desc(sa + ks * 256, 128, SBO), desc(smem_addr(sR) + ks * 256, 128, SBO), id, ch > 0 || ks > 0);
      commit(&sfree[ch % MS]);
      mmas = ch + 1;
      if (issued < nch) {
        ok = mbar_wait(&sfree[ch % MS], (ch / MS) & 1);  // this slot's MMAs have read it
        if (ok) load(issued++);
      }
    }
    if (ok) {
      commit(&accb);
    } else {
      for (int u = issued > MS ? issued - MS : 0; u < issued; ++u) mbar_wait(&full[u % MS], (u / MS) & 1);
      if (mmas > 0) mbar_wait(&sfree[(mmas - 1) % MS], ((mmas - 1) / MS) & 1);
      atomicExch(err, 1);
      mbar_arrive(&accb);  // release the other threads (they skip the read-back)
    }
  }
  {
    const bool w = mbar_wait(&accb, 0);
    ok = __syncthreads_and(ok && w);
  }
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
      // columns are (o, re/im) interleaved; write the C real parts, then the C imaginary parts,
      // each run of 8 outputs o at its place in the instance's stage-1 operand image
      const uint32_t LBO_A1 = (g.MP / 8) * 128;
      uint8_t* img = reinterpret_cast<uint8_t*>(chat + (size_t)b * g.MP * g.KXP);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        // run o0 of (k2, k = 2j + t) starts at mnmajor_off(k2 C + o0, k) = base + (o0 / 8) 128
        const uint32_t base = mnmajor_off(k2 * C, 2 * j + t, LBO_A1, 128);
        uint4* dst = reinterpret_cast<uint4*>(img + base);
#pragma unroll
        for (int o0 = 0; o0 < C; o0 += 8)
          dst[o0] = make_uint4(pack2(val[2 * o0 + t], val[2 * o0 + 2 + t], bf16),
                               pack2(val[2 * o0 + 4 + t], val[2 * o0 + 6 + t], bf16),
                               pack2(val[2 * o0 + 8 + t], val[2 * o0 + 10 + t], bf16),
                               pack2(val[2 * o0 + 12 + t], val[2 * o0 + 14 + t], bf16));
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, TCOLS);
}

struct SynArgs {
  TcGeom g;
  int B;
  int bf16;
  int din, dout;          // input / output tile ring depths
  const int* active;
  const uint16_t* vin;    // layer input, tile-major
  uint16_t* vout;         // layer output, tile-major
  const uint16_t* chat;   // [B] images MP x KXP of the stage-1 operand (MN-major)
  const uint16_t* W;      // C x C image (K-major)
  const float* bias;      // [C]
  const uint16_t* H;      // [N / SPC] images 2SPC x KXP (K-major)
  const uint16_t* Asyn;   // images 128 x KSYN (K-major): one (N < 128) or one per 128-row q tile
  int activate;
  uint16_t* hsave;        // training: pre-activations, tile-major (or null)
  // decoder (last layer)
  int project;
  const uint16_t* P1;     // C x C image (K-major)
  const float* p1;
  const float* p2;
  const float* p2b;
  const double* rms;
  double hh;              // h^2 output scale
  const double* kinv;     // [B][N][N] 1/k, the pointwise output scale of output_scale 1 (else null)
  double* z;              // [B][N][N]
  int* err;
};

// Synthesis + pointwise + bias + activation (+ decoder) for one grid-column chunk of one instance.
//
// Warp-specialised: warps 0-7 (256 threads) are the epilogue; warps w and w+4 read the same
// 32 TMEM lanes (quadrant w % 4) and split the columns (U read-back) and the channels (tile
// epilogue) between them. Lane 0 of warp 8 issues every MMA and lane 0 of warp 9 every bulk
// copy into shared memory (warp 10 has no role left).
// The roles meet only on mbarriers; four TMEM accumulators let the MMAs run up to three
// tiles ahead of the epilogue, so that their latency is hidden.
//
// Data movement: the chunk-invariant operands arrive by one bulk copy each. The activation
// tiles (128 grid points x C channels, tile-major, so each is one contiguous block already in
// the K-major operand layout) stream through a ring of din input slots, each filled by one
// bulk copy and released as soon as its MMA has completed. A hidden layer's epilogue writes
// its tile rows straight to the tile-major output (consecutive threads, consecutive 16-byte
// rows: coalesced), which leaves the copy engine to the loads; the last layer writes them into
// a ring of dout output slots (same layout) read by the decoder MMA. For N >= 128 the chunk's
// tiles are visited row block by row block (tile t: q tile t / SPC, column t % SPC).
constexpr int kSynEpi = 256;                 // epilogue threads
constexpr int kSynThreads = kSynEpi + 96;    // + the MMA, load and store warps
constexpr int kSynMaxIn = 8, kSynMaxOut = 2;
constexpr int kSynAcc = 4;                   // TMEM tile accumulators
template <int C>
__global__ void __launch_bounds__(kSynThreads, 2) tc_synthesis_kernel(SynArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // barriers: full[s] input tile copied in; infree[s] its MMA done; accfull[a] accumulator a
  // ready; accempty[a] accumulator a read back (8 warp arrivals); outready[o] output slot o
  // written (8); outfree[o] output slot o read by its store or decoder MMA; prob prologue
  // copies; s1b stage 1 done; ubar U staged in shared memory (8); decdone decoder MMA done
  __shared__ uint64_t full[kSynMaxIn], infree[kSynMaxIn], outready[kSynMaxOut], outfree[kSynMaxOut];
  __shared__ uint64_t accfull[kSynAcc], accempty[kSynAcc], prob, s1b, ubar, decdone[2];
  __shared__ uint32_t tbase_s;
  const TcGeom& g = a.g;
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (tc_inactive(a.active, b)) return;
  const int N = g.N, PC = g.SPC, Ky = g.Ky, DI = a.din, DO = a.dout;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool bf16 = a.bf16;
  const int p0 = chunk * PC;
  // shared layout
  const uint32_t LBO_A1 = (g.MP / 8) * 128;  // MN-major: K-direction core-matrix stride
  const uint32_t SBO_B = g.KB * 16, SBO_S = g.KSYN * 16, SBO_C = C * 16;
  constexpr uint32_t TB = 128 * C * 2, LBO_T = 128 * 16;
  const uint32_t SB = 128 * g.KSYN * 2;
  const uint32_t SL = TB + (N >= 128 ? SB : 0);  // input slot: tile, then (N >= 128) its table rows
  const uint32_t bytesA1 = g.MP * g.KXP * 2, bytesH = 2 * PC * g.KXP * 2;
  // region R0 holds the input and output rings and, at its top end (aliased with the last
  // slots until stage 1 has completed), the mixed coefficients for synthesis stage 1; the
  // input slots wholly below them are filled from the start of the block
  const uint32_t ring_bytes = DI * SL + DO * TB;
  const uint32_t r0 = bytesA1 > ring_bytes ? bytesA1 : ring_bytes;
  const uint32_t a1_off = (r0 - bytesA1) & ~1023u;
  const int early = (int)(a1_off / SL) < DI ? (int)(a1_off / SL) : DI;  // slots free during stage 1
  uint8_t* sA1 = smem + a1_off;            // MP x KXP
  uint8_t* ring = smem;                    // DI input slots of SL bytes (after stage 1)
  uint8_t* oring = smem + DI * SL;         // DO output slots of TB bytes (after stage 1)
  uint8_t* sH = smem + r0;                 // 2PC x KXP
  uint8_t* sB = sH + bytesH;               // C x KB
  uint8_t* sS = sB + C * g.KB * 2;         // 128 x KSYN (N < 128: one table for all tiles)
  uint8_t* sW = sS + (N < 128 ? SB : 0);   // C x C
  uint8_t* sP = sW + C * C * 2;            // C x C (decoder)
  constexpr uint32_t TCOLS = 256;
  if (warp == 0) tmem_alloc(&tbase_s, TCOLS);
  if (tid == kSynEpi) {
    for (int i = 0; i < DI; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&infree[i], 1);
    }
    for (int i = 0; i < DO; ++i) {
      mbar_init(&outready[i], kSynEpi / 32);
      mbar_init(&outfree[i], 1);
    }
    for (int i = 0; i < kSynAcc; ++i) {
      mbar_init(&accfull[i], 1);
      mbar_init(&accempty[i], kSynEpi / 32);
    }
    mbar_init(&prob, 1);
    mbar_init(&s1b, 1);
    mbar_init(&ubar, kSynEpi / 32);
    mbar_init(&decdone[0], 1);
    mbar_init(&decdone[1], 1);
  }
  // zero the K tail of the staged U columns (read by padded synthesis K steps)
  const int kvalid = PC * 2 * Ky;
  for (int idx = tid; idx < C * ((g.KB - (kvalid & ~7)) / 8); idx += kSynThreads) {
    const int nk = (g.KB - (kvalid & ~7)) / 8;
    const int row = idx / nk, kc = (kvalid & ~7) / 8 + idx % nk;
    *reinterpret_cast<uint4*>(sB + kmajor_off(row, kc * 8, 128, SBO_B)) = make_uint4(0, 0, 0, 0);
  }
  fence_smem_to_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = tbase_s;
  const uint32_t tU = tbase;                   // (MP/128) x 2PC columns (stage 1)
  const uint32_t tD = tbase;                   // kSynAcc x C tile accumulators (reuse U's columns)
  const uint32_t tE = tbase + kSynAcc * C;     // 2 x C decoder accumulators (tile parity)
  const int utiles = g.MP / 128;
  const int ntiles = (N < 128) ? PC / g.PT : PC * (N / 128);
  const size_t inst_tiles = (size_t)N * N / 128;
  // tile-major index of tile t of this chunk
  auto tile_index = [&](int t) -> size_t {
    const size_t tau = (N < 128) ? (size_t)(p0 / g.PT + t) : (size_t)(t / PC) * N + p0 + t % PC;
    return (size_t)b * inst_tiles + tau;
  };
  bool ok = true;
  if (warp == kSynEpi / 32) {
    // ================================ MMA issuer (one lane) ============================
    if (lane == 0) {
      int mmas = 0, decs = 0;
      bool s1_pending = false;
      const uint32_t idD = idesc_f16(128, C, bf16);
      // descriptors with the address field advanced per slot / K step (address >> 4 in the
      // low bits, no carry: shared addresses are below 256 KB)
      const uint64_t dX0 = desc(smem_addr(ring), LBO_T, 128);
      const uint64_t dO0 = desc(smem_addr(oring), LBO_T, 128);
      const uint64_t dW0 = desc(smem_addr(sW), 128, SBO_C);
      const uint64_t dS0 = desc(smem_addr(N < 128 ? sS : ring + TB), 128, SBO_S);
      const uint64_t dB0 = desc(smem_addr(sB), 128, SBO_B);
      const uint64_t dP0 = desc(smem_addr(sP), 128, SBO_C);
      const int ksyn = g.KSYN / 16;
      auto mma_tile = [&](int t) {
        const int acc = t % kSynAcc;
        const uint64_t slot = (uint64_t)(((t % DI) * SL) >> 4);
#pragma unroll
        for (int ks = 0; ks < C / 16; ++ks)
          mma(tD + acc * C, dX0 + slot + ks * (2 * LBO_T >> 4), dW0 + ks * 16, idD, ks > 0);
        const int kb0 = (N < 128) ? t * g.PT * 2 * Ky : (t % PC) * 2 * Ky;
        const uint64_t dS = dS0 + (N < 128 ? 0 : slot), dB = dB0 + (uint64_t)((kb0 / 8) * 8);
        for (int ks = 0; ks < ksyn; ++ks) mma(tD + acc * C, dS + ks * 16, dB + ks * 16, idD, true);
        commit(&accfull[acc]);
        commit(&infree[t % DI]);
      };
      // decoder MMA of tile u once its (GELU'd) layer output is in its output slot
      auto decode = [&](int u) -> bool {
        if (!mbar_wait(&outready[u % DO], (u / DO) & 1)) return false;
        fence_after_sync();
        const uint64_t slot = (uint64_t)(((u % DO) * TB) >> 4);
#pragma unroll
        for (int ks = 0; ks < C / 16; ++ks)
          mma(tE + (u & 1) * C, dO0 + slot + ks * (2 * LBO_T >> 4), dP0 + ks * 16, idD, ks > 0);
        commit(&decdone[u & 1]);
        commit(&outfree[u % DO]);
        decs = u + 1;
        return true;
      };
      // synthesis stage 1: U = c' H^T for the chunk
      ok = mbar_wait(&prob, 0);
      if (ok) {
        const uint32_t id = idesc_f16(128, 2 * PC, bf16, true, false);
        for (int ut = 0; ut < utiles; ++ut)
          for (int ks = 0; ks < g.KXP / 16; ++ks)
            mma(tU + ut * 2 * PC, desc(smem_addr(sA1) + ut * 16 * 128 + ks * 2 * LBO_A1, LBO_A1, 128),
                desc(smem_addr(sH) + ks * 256, 128, g.KXP * 16), id, ks > 0);
        commit(&s1b);
        s1_pending = true;
        ok = mbar_wait(&ubar, 0);  // U read back and staged in sB by the epilogue warps
        if (ok) s1_pending = false;
        fence_after_sync();
      }
      constexpr int LAG = 2;  // decoder of tile t - LAG issued after tile t's MMAs
      for (int t = 0; t < ntiles && ok; ++t) {
        ok = mbar_wait(&full[t % DI], (t / DI) & 1);
        if (ok && t >= kSynAcc) ok = mbar_wait(&accempty[t % kSynAcc], ((t / kSynAcc) - 1) & 1);
        if (!ok) break;
        fence_after_sync();
        mma_tile(t);
        mmas = t + 1;
        if (a.project && t >= LAG) ok = decode(t - LAG);
      }
      for (int u = decs; ok && a.project && u < ntiles; ++u) ok = decode(u);
      if (!ok) {
        // error path: let the MMAs this block started finish (bounded) before the block
        // releases its tensor memory
        if (s1_pending) mbar_wait(&s1b, 0);
        for (int u = mmas > kSynAcc ? mmas - kSynAcc : 0; u < mmas; ++u)
          mbar_wait(&accfull[u % kSynAcc], (u / kSynAcc) & 1);
        if (decs > 0) mbar_wait(&decdone[(decs - 1) & 1], ((decs - 1) >> 1) & 1);
        atomicExch(a.err, 1);
      }
    }
  } else if (warp == kSynEpi / 32 + 1) {
    // ================================ load issuer (one lane) ===========================
    if (lane == 0) {
      int loads = 0;
      bool pro_pending = false;
      auto load_tile = [&](int t) {
        const int s = t % DI;
        uint8_t* dst = ring + s * SL;
        mbar_expect_tx(&full[s], SL);
        bulk_g2s(dst, a.vin + tile_index(t) * 128 * C, TB, &full[s]);
        if (N >= 128) bulk_g2s(dst + TB, a.Asyn + (size_t)(t / PC) * 128 * g.KSYN, SB, &full[s]);
        loads = t + 1;
      };
      // constant operands and the first input tiles (the layer input was written three
      // kernels back) before the wait; the mixed coefficients come from the kernel just before
      mbar_expect_tx(&prob, bytesA1 + bytesH + C * C * 2 * (a.project ? 2 : 1) + (N < 128 ? SB : 0));
      bulk_g2s(sH, a.H + (size_t)chunk * 2 * PC * g.KXP, bytesH, &prob);
      bulk_g2s(sW, a.W, C * C * 2, &prob);
      if (a.project) bulk_g2s(sP, a.P1, C * C * 2, &prob);
      if (N < 128) bulk_g2s(sS, a.Asyn, SB, &prob);
      while (loads < ntiles && loads < early) load_tile(loads);
      pdl_wait();
      pdl_trigger();
      bulk_g2s(sA1, a.chat + (size_t)b * g.MP * g.KXP, bytesA1, &prob);
      ok = mbar_wait(&prob, 0);
      pro_pending = !ok;
      if (ok) ok = mbar_wait(&s1b, 0);  // stage 1 has read sA1: the rings may overwrite it
      if (ok)
        while (loads < ntiles && loads < DI) load_tile(loads);
      // refill the input slot of tile u as soon as its MMA has read it
      for (int u = 0; u + DI < ntiles && ok; ++u) {
        ok = mbar_wait(&infree[u % DI], (u / DI) & 1);
        if (ok) load_tile(u + DI);
      }
      if (!ok) {
        // error path: let every copy this block started finish (bounded)
        if (pro_pending) mbar_wait(&prob, 0);
        for (int u = loads > DI ? loads - DI : 0; u < loads; ++u) mbar_wait(&full[u % DI], (u / DI) & 1);
        atomicExch(a.err, 1);
      }
    }
  } else if (warp == kSynEpi / 32 + 2) {
    // ================================ (idle warp) =====================================
    // hidden layers store straight from the epilogue; the last layer's output slots are read
    // by the decoder MMA
  } else {
    // ================================ epilogue (256 threads) ===========================
    pdl_wait();  // (before its global writes)
    const int quad = warp & 3, half = warp >> 2;  // TMEM lane quadrant, channel/column half
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    ok = mbar_wait(&s1b, 0);
    fence_after_sync();
    if (ok) {
      // U lane (k2, c), columns (p, t') -> sB[c][(p, k2, t')]
      for (int ut = 0; ut < utiles; ++ut) {
        const int row = ut * 128 + quad * 32 + lane;
        const int k2 = row / C, c = row % C;
        if (PC % 16 == 0) {
          for (int c0 = half * PC; c0 < (half + 1) * PC; c0 += 16) {
            float val[16];
            tmem_ld16(tU + ut * 2 * PC + c0 + lane_off, val);
            if (row < Ky * C) {
#pragma unroll
              for (int i = 0; i < 16; i += 2) {
                const int pl = (c0 + i) >> 1;
                *reinterpret_cast<uint32_t*>(sB + kmajor_off(c, pl * 2 * Ky + 2 * k2, 128, SBO_B)) =
                    pack2(val[i], val[i + 1], bf16);
              }
            }
          }
        } else {
          // 8-column chunks (narrow launch shape): each half reads its 8 of U's 16 columns
          const int c0 = half * PC;
          float val[8];
          tmem_ld8(tU + ut * 2 * PC + c0 + lane_off, val);
          if (row < Ky * C) {
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
              const int pl = (c0 + i) >> 1;
              *reinterpret_cast<uint32_t*>(sB + kmajor_off(c, pl * 2 * Ky + 2 * k2, 128, SBO_B)) =
                  pack2(val[i], val[i + 1], bf16);
            }
          }
        }
      }
      fence_smem_to_async();
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ubar);
    }
    // Thread tid owns tile row m = tid % 128 of every tile: its grid point within the tile is
    // fixed, so the row's (q, column offset) are computed once.
    const int m = tid & 127;
    const int own_pl = (N < 128) ? m / N : 0;     // column within the tile (N < 128)
    const int own_q = (N < 128) ? m % N : m;      // row (N < 128) or row within the q-tile
    constexpr int CH = C / 2;  // channels per thread in the epilogue
    const int cbase = half * CH;
    float bias[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) bias[c] = a.bias[cbase + c];
    // Last layer: the MMA warp multiplies tile u's output slot by the decoder weights into
    // accumulator u & 1; the epilogue half u & 1 (warps 0-3 even tiles, 4-7 odd tiles) finishes
    // tile u (GELU, -> 1, output scale, z) from all C columns of its TMEM lanes, after it has
    // written tile u + 1's slot, so that the decoder MMA's latency overlaps that work and the
    // halves exchange nothing. A thread's read of accumulator u & 1 precedes its arrival on tile
    // u + 2's slot, which the MMA of decoder u + 2 (the accumulator's next use) waits for.
    const double zscale = a.project ? a.rms[b] * a.hh : 0.0;
    auto decoder_part = [&](int u, bool okd) -> bool {
      if (half != (u & 1)) return okd;
      if (okd) {
        okd = mbar_wait(&decdone[u & 1], (u >> 1) & 1);
        fence_after_sync();
      }
      if (okd) {
        float zt = a.p2b[0];
#pragma unroll
        for (int c0 = 0; c0 < C; c0 += 16) {
          float val[16];
          tmem_ld16(tE + (u & 1) * C + c0 + lane_off, val);
#pragma unroll
          for (int i = 0; i < 16; ++i) zt = fmaf(a.p2[c0 + i], gelu16(val[i] + a.p1[c0 + i]), zt);
        }
        int q, p;
        if (N < 128) {
          q = own_q;
          p = p0 + u * g.PT + own_pl;
        } else {
          p = p0 + u % PC;
          q = (u / PC) * 128 + own_q;
        }
        const size_t zi = ((size_t)b * N + q) * N + p;
        a.z[zi] = (a.kinv ? zscale * a.kinv[zi] : zscale) * (double)zt;
      }
      fence_before_sync();
      return okd;
    };
    for (int t = 0; t < ntiles; ++t) {
      if (ok) {
        ok = mbar_wait(&accfull[t % kSynAcc], (t / kSynAcc) & 1);
        fence_after_sync();
      }
      float h[CH];
      if (ok) {
        const uint32_t col = tD + (t % kSynAcc) * C + cbase + lane_off;
        if constexpr (CH == 16) {
          tmem_ld16(col, h);
        } else {
          tmem_ld8(col, h);
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accempty[t % kSynAcc]);
#pragma unroll
        for (int i = 0; i < CH; ++i) h[i] += bias[i];
        if (a.hsave) {
          // training: the pre-activation of this tile row, tile-major like the output
          uint8_t* dsth = reinterpret_cast<uint8_t*>(a.hsave + tile_index(t) * 128 * C) + m * 16;
#pragma unroll
          for (int c0 = 0; c0 < CH; c0 += 8)
            *reinterpret_cast<uint4*>(dsth + ((cbase + c0) / 8) * LBO_T) =
                make_uint4(pack2(h[c0], h[c0 + 1], bf16), pack2(h[c0 + 2], h[c0 + 3], bf16),
                           pack2(h[c0 + 4], h[c0 + 5], bf16), pack2(h[c0 + 6], h[c0 + 7], bf16));
        }
        if (a.activate) {
#pragma unroll
          for (int i = 0; i < CH; ++i) h[i] = gelu16(h[i]);
        }
        // the output slot's previous tile (t - DO) has been decoded
        if (a.project && t >= DO) ok = mbar_wait(&outfree[t % DO], ((t / DO) - 1) & 1);
      }
      if (ok && !a.project) {
        // hidden layer: the tile row goes straight to the tile-major output (consecutive
        // threads write consecutive 16-byte rows), leaving the copy engine to the loads
        uint8_t* dst = reinterpret_cast<uint8_t*>(a.vout + tile_index(t) * 128 * C) + m * 16;
#pragma unroll
        for (int c0 = 0; c0 < CH; c0 += 8) {
          *reinterpret_cast<uint4*>(dst + ((cbase + c0) / 8) * LBO_T) =
              make_uint4(pack2(h[c0], h[c0 + 1], bf16), pack2(h[c0 + 2], h[c0 + 3], bf16),
                         pack2(h[c0 + 4], h[c0 + 5], bf16), pack2(h[c0 + 6], h[c0 + 7], bf16));
        }
      } else if (ok) {
        uint8_t* dst = oring + (t % DO) * TB + m * 16;
#pragma unroll
        for (int c0 = 0; c0 < CH; c0 += 8) {
          *reinterpret_cast<uint4*>(dst + ((cbase + c0) / 8) * LBO_T) =
              make_uint4(pack2(h[c0], h[c0 + 1], bf16), pack2(h[c0 + 2], h[c0 + 3], bf16),
                         pack2(h[c0 + 4], h[c0 + 5], bf16), pack2(h[c0 + 6], h[c0 + 7], bf16));
        }
        fence_smem_to_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&outready[t % DO]);
      }
      // last layer: the previous tile's decoder output, whose MMA ran while this tile was finished
      if (a.project && t > 0) ok = decoder_part(t - 1, ok);
      if (!ok) break;
    }
    if (a.project && ok) decoder_part(ntiles - 1, ok);
  }
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
static size_t mix_smem(const TcGeom& g) {
  const int ms = g.nchunks < kMixSlots ? g.nchunks : kMixSlots;
  return (size_t)4 * g.C * g.C * 2 + (size_t)ms * 128 * 2 * g.C * 2;
}
// Tile rings of the synthesis kernel: the deepest input ring (2 .. kSynMaxIn slots, 2 output
// slots) that keeps two blocks per SM; kSynMaxIn + 2 (one block per SM) when none does.
static void synthesis_rings(const TcGeom& g, int& din, int& dout) {
  dout = kSynMaxOut;
  for (din = kSynMaxIn; din >= 2; --din)
    if (synthesis_bytes(g, g.SPC, din, dout) <= kSynTwoPerSm) return;
  din = kSynMaxIn;
}

// The synthesis geometry of the narrow launch shape: 8-column chunks for N < 128 (4 tiles per
// block at 64 x 64 instead of 16). The H table's chunk images of any width that is a multiple of
// 4 columns are consecutive slices of the same bytes (its rows are grouped by 8 with a fixed
// stride), so both shapes read one table.
static TcGeom narrow_geom(TcGeom g) {
  if (g.N >= 128 || g.SPC <= 8) return g;
  // analysis and mixing: 16-column chunks (half the serial m-tile steps per block, twice the
  // partial-coefficient images for the mixing to sum)
  if (g.PC > 16) {
    g.PC = 16;
    g.nchunks = g.N / g.PC;
  }
  g.SPC = 8;
  while (g.SPC % g.PT != 0) g.SPC *= 2;
  g.snchunks = g.N / g.SPC;
  g.KB = round_up(g.SPC * 2 * g.M, 16) + 16;
  return g;
}

bool tc_has_narrow(int N, const fcgno_model_desc& d) {
  if (!tc_shape_supported(N, d)) return false;
  const TcGeom g = make_geom(N, d.width, d.modes);
  return narrow_geom(g).SPC != g.SPC;
}

// The operator's 16-bit activation buffers for grid geometry g (either launch shape).
static fcgno_status ensure_acts(fcgno_model* m, const fcgno_op* op, const TcGeom& g, cudaStream_t st) {
  FCGNO_TRY(ensure_err_flag(op, st));
  TcActs& T = *op->tc_acts;
  size_t need_v, need_part, need_chat;
  tc_acts_elems(g, op->B, need_v, need_part, need_chat);
  if (T.cap_v >= need_v && T.cap_part >= need_part && T.cap_chat >= need_chat) return FCGNO_OK;
  free_acts(T);
  if (cudaMalloc(&T.va, need_v * 2) != cudaSuccess || cudaMalloc(&T.vb, need_v * 2) != cudaSuccess ||
      cudaMalloc(&T.part, need_part * 2) != cudaSuccess || cudaMalloc(&T.chat, need_chat * 2) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("tensor-core preconditioner workspace: out of device memory");
    return FCGNO_ENOMEM;
  }
  // the padding of the stage-1 operand images is never written: zero it once
  FCGNO_CUDA_TRY(cudaMemsetAsync(T.chat, 0, need_chat * 2, st));
  T.cap_v = need_v;
  T.cap_part = need_part;
  T.cap_chat = need_chat;
  m->gen++;
  return FCGNO_OK;
}

// Dynamic shared-memory limits of the three layer kernels, raised to cover both launch shapes
// of grid geometry g (wide g), so that the other shape's first (captured) launch needs no
// attribute change. A limit is raised only when a larger plan appears (not a stream operation;
// the first solve iteration runs eagerly, before any graph capture). The shared-memory carveout
// is pinned to its maximum so that two blocks of each kernel stay resident per SM; left to the
// CUDA driver it may size the carveout for one block.
template <int C>
static fcgno_status raise_smem_limits(const TcGeom& g) {
  const TcGeom gn = narrow_geom(g);
  const size_t sa_limit = std::max(analysis_smem(g), analysis_smem(gn));
  const size_t sm_limit = std::max(mix_smem(g), mix_smem(gn));
  size_t ss_limit = 0;
  for (const TcGeom& go : {g, gn}) {
    int di, dout;
    synthesis_rings(go, di, dout);
    ss_limit = std::max(ss_limit, synthesis_bytes(go, go.SPC, di, dout));
  }
  static std::mutex set_mu;  // concurrent callers on other threads share these limits
  static size_t set_sa = 0, set_ss = 0, set_sm = 0, set_sp = 0;
  std::lock_guard<std::mutex> set_lk(set_mu);
  auto raise = [](const void* fn, size_t bytes, size_t& set) -> cudaError_t {
    if (bytes <= set) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) set = bytes;
    return e;
  };
  FCGNO_CUDA_TRY(raise((const void*)tc_analysis_kernel<C>, sa_limit, set_sa));
  if (ana_pipe_ok(g)) FCGNO_CUDA_TRY(raise((const void*)tc_analysis_pipe_kernel<C>, analysis_smem(g), set_sp));
  FCGNO_CUDA_TRY(raise((const void*)tc_synthesis_kernel<C>, ss_limit, set_ss));
  FCGNO_CUDA_TRY(raise((const void*)tc_mix_kernel<C>, sm_limit, set_sm));
  return FCGNO_OK;
}

template <int C>
static fcgno_status run_tc(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms, const int* active,
                           double* z, bool fp16, cudaStream_t st, bool narrow) {
  const fcgno_model_desc& d = m->desc;
  const TcGeom g = make_geom(op->N, C, d.modes);
  const TcGeom gn = narrow_geom(g);
  const TcGeom gs = narrow ? gn : g;  // geometry of this call's launches
  const uint64_t gen0 = m->gen;
  FCGNO_TRY(ensure_prec(m, fp16, st));
  TcTables* tab = nullptr;
  FCGNO_TRY(ensure_tables(m, fp16, g, tab, st));
  // the other launch shape's tables are built in the same (eager) call, so that no table build
  // is ever captured into a replayed graph
  TcTables* tabn = nullptr;
  FCGNO_TRY(ensure_tables(m, fp16, gn, tabn, st));
  if (narrow) tab = tabn;
  if (m->gen != gen0) {
    // derived weight images or tables were just built on `st`: finish them before going on,
    // so that operators solved on other streams never read them half written. This happens
    // once per model, precision and grid, in the eager first iteration of a solve or bucket;
    // under stream capture the build kernels are captured ahead of their readers instead.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FCGNO_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (cap == cudaStreamCaptureStatusNone) FCGNO_CUDA_TRY(cudaStreamSynchronize(st));
  }
  TcPrecision& P = m->tc->prec[fp16 ? 1 : 0];
  FCGNO_TRY(ensure_acts(m, op, g, st));
  TcActs& T = *op->tc_acts;
  const int B = op->B;
  const int nbt = ceil_div(B, 128);
  BlobLayout BL = blob_layout(d);
  const bool bf16 = !fp16;
  {
    TraceScope ts("tc_lift", st);
    const int lift_blocks = (op->N / kLiftCols) * (op->N / lift_rows(op->N));
    FCGNO_CUDA_TRY(launch_chained(tc_lift_kernel<C>, dim3(lift_blocks, B), dim3(kLiftThreads), 0, st, g, r,
                                  (const float*)op->logk32, rms, active, (const float*)(m->w32 + BL.lift_w),
                                  (const float*)(m->w32 + BL.lift_b), T.va, bf16));
  }
  FCGNO_LAUNCHED();
  int din, dout;
  synthesis_rings(gs, din, dout);
  const size_t sa = analysis_smem(gs), ss = synthesis_bytes(gs, gs.SPC, din, dout), sm = mix_smem(gs);
  FCGNO_TRY(raise_smem_limits<C>(g));
  uint16_t* cur = T.va;
  uint16_t* nxt = T.vb;
  for (int l = 0; l < d.layers; ++l) {
    {
      TraceScope ts("tc_analysis", st);
      if (!narrow && ana_pipe_ok(gs)) {
        // wide shape: persistent blocks, each walking the instances of one column chunk
        FCGNO_CUDA_TRY(launch_chained(tc_analysis_pipe_kernel<C>, dim3(ana_pipe_blocks(gs, B)),
                                      dim3(kAnaPipeThreads), sa, st, gs, B, nbt, bf16, active,
                                      (const uint16_t*)cur, (const uint16_t*)tab->E2, (const uint16_t*)tab->G,
                                      T.part, T.err, 1));
      } else {
        FCGNO_CUDA_TRY(launch_chained(tc_analysis_kernel<C>, dim3(gs.nchunks, B), dim3(kAnaThreads), sa, st, gs,
                                      nbt, bf16, active, (const uint16_t*)cur, (const uint16_t*)tab->E2,
                                      (const uint16_t*)tab->G, T.part, T.err));
      }
    }
    FCGNO_LAUNCHED();
    {
      TraceScope ts("tc_mix", st);
      FCGNO_CUDA_TRY(launch_chained(tc_mix_kernel<C>, dim3(gs.nmodes, nbt), dim3(kTcThreads), sm, st, gs, B, nbt,
                                    bf16, active, (const uint16_t*)T.part, (const uint16_t*)P.Rr[l], T.chat,
                                    T.err));
    }
    FCGNO_LAUNCHED();
    SynArgs s{};
    s.vin = cur;
    s.vout = nxt;
    s.g = gs;
    s.B = B;
    s.bf16 = bf16;
    // hidden layers store straight from the epilogue: their input ring also takes the
    // output slots' bytes (same shared-memory size)
    const bool last = l == d.layers - 1;
    const size_t slot_in = (size_t)128 * C * 2 + (gs.N >= 128 ? (size_t)128 * gs.KSYN * 2 : 0);
    s.din = last ? din : std::min<int>(kSynMaxIn, (int)(((size_t)din * slot_in + (size_t)dout * 128 * C * 2) / slot_in));
    s.dout = last ? dout : 0;
    s.active = active;
    s.chat = T.chat;
    s.W = P.W[l];
    s.bias = m->w32 + BL.b[l];
    s.H = tab->H;
    s.Asyn = tab->Asyn;
    s.activate = l < d.layers - 1;
    s.project = l == d.layers - 1;
    s.P1 = P.P1;
    s.p1 = m->w32 + BL.proj1_b;
    s.p2 = m->w32 + BL.proj2_w;
    s.p2b = m->w32 + BL.proj2_b;
    s.rms = rms;
    s.hh = 1.0 / ((double)(op->N + 1) * (op->N + 1));
    s.kinv = d.output_scale ? op->kinv : nullptr;
    s.z = z;
    s.err = T.err;
    {
      TraceScope ts("tc_synthesis", st);
      FCGNO_CUDA_TRY(launch_chained(tc_synthesis_kernel<C>, dim3(gs.snchunks, B), dim3(kSynThreads), ss, st, s));
    }
    FCGNO_LAUNCHED();
    std::swap(cur, nxt);
  }
  return FCGNO_OK;
}

size_t tc_acts_bytes(int N, int B, const fcgno_model_desc& d) {
  if (!tc_shape_supported(N, d)) return 0;
  const TcGeom g = make_geom(N, d.width, d.modes);
  size_t v, part, chat;
  tc_acts_elems(g, B, v, part, chat);
  return 2 * (2 * v + part + chat) + sizeof(int);  // 16-bit elements; the timeout flag
}

bool tc_shape_supported(int N, const fcgno_model_desc& d) {
  return geom_supported(N, d.width, d.modes, d.proj_width);
}

const char* tc_shape_rule() {
  return "the 16-bit preconditioner supports width 16 or 32 (proj_width = width), modes <= 16 and "
         "N in {32, 64} or a multiple of 128";
}

fcgno_status no_apply_tc(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms, const int* active,
                         double* z, bool fp16, cudaStream_t st, bool narrow) {
  const fcgno_model_desc& d = m->desc;
  if (!tc_shape_supported(op->N, d)) {
    set_last_error(tc_shape_rule());
    return FCGNO_EINVAL;
  }
  if (d.width == 16) return run_tc<16>(m, op, r, rms, active, z, fp16, st, narrow);
  return run_tc<32>(m, op, r, rms, active, z, fp16, st, narrow);
}

// ------------------------------------ training (BF16) ----------------------------------
// The training step of Eq. (11) with BF16 operands and FP32 accumulation (Section 2.4.1):
// the forward runs the tensor-core layers above and keeps every layer's input and
// pre-activation (tile-major BF16) and its analysis output; the backward runs the adjoint of
// each Fourier layer's data path on the same three kernels, with the adjoint tables and the
// transposed weight images:
//   analysis, adjoint tables, on gh  -> g'    = w(k2) sum_x gh(x) e^{-i theta_k(x)}
//   mixing with the transposed real forms of R -> gc = R^H g'   (per mode)
//   synthesis with W^T, the adjoint Asyn, zero bias, no activation
//                                     -> gv_in = W^T gh + (1/n) Re sum_k gc e^{+i theta_k(x)}
// The weight gradients are FP32 reductions on CUDA cores over the saved tiles converted to
// FP32 (the per-mode one needs the analysis outputs of the forward and of the backward,
// summed over column chunks here). The host side of the step composes these pieces with the
// loss and the decoder.

__host__ __device__ __forceinline__ void act_point_of(const TcGeom& g, int tau, int m, int& q, int& p) {
  if (g.N < 128) {
    p = tau * g.PT + m / g.N;
    q = m % g.N;
  } else {
    q = (tau / g.N) * 128 + m;
    p = tau % g.N;
  }
}

__device__ __forceinline__ void unpack_bf16x8(uint4 w, float* f) {
  const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[i]));
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}

// One thread per (tile row, 8-channel group); consecutive threads read consecutive 16-byte
// rows of a tile. Returns false past the end. Sets the 16-bit element offset of the row group
// in the tile-major buffer and the FP32 offset of the same 8 channels in [B][N][N][C].
__device__ __forceinline__ bool tile_row_group(const TcGeom& g, int B, size_t i, size_t& toff, size_t& foff) {
  const int C = g.C, CG = C / 8;
  const size_t n = (size_t)g.N * g.N, tiles = n / 128;
  if (i >= (size_t)B * n * CG) return false;
  const int m = (int)(i % 128);
  const size_t rest = i / 128;
  const int cg = (int)(rest % CG);
  const size_t tile = rest / CG;
  const int b = (int)(tile / tiles), tau = (int)(tile % tiles);
  int q, p;
  act_point_of(g, tau, m, q, p);
  toff = tile * 128 * C + (size_t)cg * 1024 + (size_t)m * 8;
  foff = ((size_t)b * n + (size_t)q * g.N + p) * C + cg * 8;
  return true;
}

// BF16 tile-major activations -> FP32 [B][N][N][C]
__global__ void tc_tile_to_f32_kernel(TcGeom g, int B, const uint16_t* __restrict__ v, float* __restrict__ out) {
  size_t toff, foff;
  if (!tile_row_group(g, B, blockIdx.x * (size_t)blockDim.x + threadIdx.x, toff, foff)) return;
  float f[8];
  unpack_bf16x8(*reinterpret_cast<const uint4*>(v + toff), f);
  float4* o = reinterpret_cast<float4*>(out + foff);
  o[0] = make_float4(f[0], f[1], f[2], f[3]);
  o[1] = make_float4(f[4], f[5], f[6], f[7]);
}

// gh = gv * GELU'(h) (or gv where the layer has no activation, h null), from gv given in FP32
// [B][N][N][C] (gv32) or BF16 tile-major (gvt); written in both forms. GELU' is the derivative
// of the exact (erf) GELU at the saved BF16 pre-activation.
__global__ void tc_act_bwd_kernel(TcGeom g, int B, const float* __restrict__ gv32, const uint16_t* __restrict__ gvt,
                                  const uint16_t* __restrict__ h, float* __restrict__ gh32,
                                  uint16_t* __restrict__ ght) {
  size_t toff, foff;
  if (!tile_row_group(g, B, blockIdx.x * (size_t)blockDim.x + threadIdx.x, toff, foff)) return;
  float gv[8];
  if (gv32) {
    const float4 a = reinterpret_cast<const float4*>(gv32 + foff)[0];
    const float4 c = reinterpret_cast<const float4*>(gv32 + foff)[1];
    gv[0] = a.x; gv[1] = a.y; gv[2] = a.z; gv[3] = a.w;
    gv[4] = c.x; gv[5] = c.y; gv[6] = c.z; gv[7] = c.w;
  } else {
    unpack_bf16x8(*reinterpret_cast<const uint4*>(gvt + toff), gv);
  }
  if (h) {
    float hv[8];
    unpack_bf16x8(*reinterpret_cast<const uint4*>(h + toff), hv);
#pragma unroll
    for (int i = 0; i < 8; ++i) gv[i] *= gelu_grad_f(hv[i]);
  }
  float4* o = reinterpret_cast<float4*>(gh32 + foff);
  o[0] = make_float4(gv[0], gv[1], gv[2], gv[3]);
  o[1] = make_float4(gv[4], gv[5], gv[6], gv[7]);
  *reinterpret_cast<uint4*>(ght + toff) = make_uint4(pack2(gv[0], gv[1], true), pack2(gv[2], gv[3], true),
                                                    pack2(gv[4], gv[5], true), pack2(gv[6], gv[7], true));
}

// Analysis partial-coefficient images (mode x column chunk x block of 128 instances, rows =
// instances, K = (c, re/im)) summed over the column chunks in FP32: out[b][mode][c] complex.
__global__ void tc_part_to_cx_kernel(TcGeom g, int B, int nbt, const uint16_t* __restrict__ part,
                                     float* __restrict__ out) {
  const int C = g.C;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)B * g.nmodes * C) return;
  const int c = (int)(i % C), mode = (int)((i / C) % g.nmodes), b = (int)(i / ((size_t)C * g.nmodes));
  const int bt = b / 128, br = b % 128;
  const size_t img = (size_t)128 * 2 * C;
  const uint32_t off = kmajor_off(br, 2 * c, 128, 2 * C * 16) / 2;  // (re, im) adjacent
  float re = 0.f, im = 0.f;
  for (int ch = 0; ch < g.nchunks; ++ch) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(part + (((size_t)mode * g.nchunks + ch) * nbt + bt) * img + off);
    const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    re += t.x;
    im += t.y;
  }
  out[2 * i] = re;
  out[2 * i + 1] = im;
}

// Bytes of one operator's BF16 training state (TcTrainBufs) for `layers` layers.
static size_t train_bufs_layout(const TcGeom& g, int B, int layers, bool recompute, size_t* offs) {
  const size_t img = (size_t)B * g.N * g.N * g.C * 2;
  size_t v, part, chat;
  tc_acts_elems(g, B, v, part, chat);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) / 256 * 256;
    return at;
  };
  int k = 0;
  for (int l = 0; l <= layers; ++l) offs[k++] = take(img);           // v
  const int nh = recompute ? (layers > 1 ? 1 : 0) : layers - 1;
  for (int l = 0; l < nh; ++l) offs[k++] = take(img);                // h
  offs[k++] = take(img);                                             // gh
  offs[k++] = take(img);                                             // gv
  offs[k++] = take(part * 2);                                        // partb
  offs[k++] = take((size_t)B * g.nmodes * g.C * 2 * sizeof(float));  // gspec
  offs[k++] = take((size_t)g.C * sizeof(float));                     // zero
  return o;
}

static fcgno_status ensure_train_bufs(const fcgno_op* op, const TcGeom& g, int layers, bool recompute,
                                      cudaStream_t st) {
  TcTrainBufs& tb = op->tc_acts->train;
  size_t offs[2 * 16 + 8];
  const size_t bytes = train_bufs_layout(g, op->B, layers, recompute, offs);
  if (tb.base && tb.bytes == bytes && tb.recompute == recompute) return FCGNO_OK;
  if (tb.base) cudaFree(tb.base);
  tb = TcTrainBufs{};
  if (cudaMalloc(&tb.base, bytes) != cudaSuccess) {
    cudaGetLastError();
    tb.base = nullptr;
    set_last_error("BF16 training workspace: out of device memory");
    return FCGNO_ENOMEM;
  }
  tb.bytes = bytes;
  uint8_t* b = (uint8_t*)tb.base;
  int k = 0;
  for (int l = 0; l <= layers; ++l) tb.v[l] = (uint16_t*)(b + offs[k++]);
  const int nh = recompute ? (layers > 1 ? 1 : 0) : layers - 1;
  for (int l = 0; l < nh; ++l) tb.h[l] = (uint16_t*)(b + offs[k++]);
  tb.recompute = recompute;
  tb.gh = (uint16_t*)(b + offs[k++]);
  tb.gv = (uint16_t*)(b + offs[k++]);
  tb.partb = (uint16_t*)(b + offs[k++]);
  tb.gspec = (float*)(b + offs[k++]);
  tb.zero = (float*)(b + offs[k++]);
  FCGNO_CUDA_TRY(cudaMemsetAsync(tb.zero, 0, sizeof(float) * g.C, st));
  return FCGNO_OK;
}

size_t tc_train_bytes(int N, int B, const fcgno_model_desc& d, bool recompute) {
  if (!tc_shape_supported(N, d)) return 0;
  size_t offs[2 * 16 + 8];
  return train_bufs_layout(make_geom(N, d.width, d.modes), B, d.layers, recompute, offs);
}

// Whether a BF16 training step on this operator rebuilds its pre-activations: mode 1 always,
// 2 never, 0 when keeping the L - 1 pre-activation images would take more than 2 GiB.
bool tc_train_recompute(const fcgno_model* m, const fcgno_op* op) {
  if (m->train_recompute == 1) return true;
  if (m->train_recompute == 2) return false;
  const size_t img = (size_t)op->B * op->n * m->desc.width * 2;
  return img * (size_t)(m->desc.layers - 1) > ((size_t)2 << 30);
}

// One synthesis launch of the hidden-layer kind (the epilogue stores the tile rows itself).
template <int C>
static fcgno_status launch_syn_hidden(const TcGeom& g, const fcgno_op* op, const uint16_t* vin, uint16_t* vout,
                                      const uint16_t* chat, const uint16_t* W, const float* bias,
                                      const TcTables* tab, int activate, uint16_t* hsave, cudaStream_t st) {
  int din, dout;
  synthesis_rings(g, din, dout);
  const size_t ss = synthesis_bytes(g, g.SPC, din, dout);
  const size_t slot_in = (size_t)128 * C * 2 + (g.N >= 128 ? (size_t)128 * g.KSYN * 2 : 0);
  SynArgs s{};
  s.g = g;
  s.B = op->B;
  s.bf16 = 1;
  s.din = std::min<int>(kSynMaxIn, (int)(((size_t)din * slot_in + (size_t)dout * 128 * C * 2) / slot_in));
  s.dout = 0;
  s.active = nullptr;
  s.vin = vin;
  s.vout = vout;
  s.chat = chat;
  s.W = W;
  s.bias = bias;
  s.H = tab->H;
  s.Asyn = tab->Asyn;
  s.activate = activate;
  s.hsave = hsave;
  s.project = 0;
  s.err = op->tc_acts->err;
  FCGNO_CUDA_TRY(launch_chained(tc_synthesis_kernel<C>, dim3(g.snchunks, op->B), dim3(kSynThreads), ss, st, s));
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

template <int C>
static fcgno_status launch_ana(const TcGeom& g, const fcgno_op* op, const uint16_t* v, const TcTables* tab,
                               uint16_t* part, cudaStream_t st) {
  FCGNO_CUDA_TRY(launch_chained(tc_analysis_kernel<C>, dim3(g.nchunks, op->B), dim3(kAnaThreads), analysis_smem(g),
                                st, g, ceil_div(op->B, 128), true, (const int*)nullptr, v, (const uint16_t*)tab->E2,
                                (const uint16_t*)tab->G, part, op->tc_acts->err));
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

template <int C>
static fcgno_status launch_mixing(const TcGeom& g, const fcgno_op* op, const uint16_t* part, const uint16_t* Rr,
                                  uint16_t* chat, cudaStream_t st) {
  const int nbt = ceil_div(op->B, 128);
  FCGNO_CUDA_TRY(launch_chained(tc_mix_kernel<C>, dim3(g.nmodes, nbt), dim3(kTcThreads), mix_smem(g), st, g, op->B,
                                nbt, true, (const int*)nullptr, part, Rr, chat, op->tc_acts->err));
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

static fcgno_status part_to_cx(const TcGeom& g, const fcgno_op* op, const uint16_t* part, float* out,
                               cudaStream_t st) {
  const size_t total = (size_t)op->B * g.nmodes * g.C;
  tc_part_to_cx_kernel<<<ceil_div(total, 256), 256, 0, st>>>(g, op->B, ceil_div(op->B, 128), part, out);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

fcgno_status tc_train_begin(fcgno_model* m, const fcgno_op* op, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  if (!tc_shape_supported(op->N, d)) {
    set_last_error(tc_shape_rule());
    return FCGNO_EINVAL;
  }
  const TcGeom g = make_geom(op->N, d.width, d.modes);
  // weight images from the current master blob (the optimiser changes it between steps)
  const bool had = m->tc && m->tc->prec[0].built;
  FCGNO_TRY(ensure_prec(m, false, st));
  TcPrecision& P = m->tc->prec[0];
  if (had) FCGNO_TRY(cast_images(m, P, true, st));
  const int C = d.width, nmodes = g.nmodes;
  BlobLayout BL = blob_layout(d);
  if (P.WT.empty()) {
    P.WT.assign(d.layers, nullptr);
    P.RrT.assign(d.layers, nullptr);
    for (int l = 0; l < d.layers; ++l) {
      FCGNO_CUDA_TRY(cudaMalloc(&P.WT[l], sizeof(uint16_t) * C * C));
      FCGNO_CUDA_TRY(cudaMalloc(&P.RrT[l], sizeof(uint16_t) * (size_t)nmodes * 4 * C * C));
    }
  }
  const size_t tot = (size_t)nmodes * 4 * C * C;
  for (int l = 0; l < d.layers; ++l) {
    tc_cast_image_kernel<<<ceil_div(C * C, 256), 256, 0, st>>>(C, C, m->w32 + BL.w[l], P.WT[l], true, true);
    FCGNO_LAUNCHED();
    tc_rr_kernel<<<ceil_div(tot, 256), 256, 0, st>>>(C, nmodes, m->w32 + BL.r[l], P.RrT[l], true, true);
    FCGNO_LAUNCHED();
  }
  TcTables* tab = nullptr;
  FCGNO_TRY(ensure_tables(m, false, g, tab, st));
  FCGNO_TRY(ensure_tables(m, false, g, tab, st, true));
  FCGNO_TRY(ensure_acts(m, op, g, st));
  FCGNO_TRY(ensure_train_bufs(op, g, d.layers, tc_train_recompute(m, op), st));
  if (C == 16) return raise_smem_limits<16>(g);
  return raise_smem_limits<32>(g);
}

template <int C>
static fcgno_status train_forward(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms,
                                  float* const* cx, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  const TcGeom g = make_geom(op->N, C, d.modes);
  TcPrecision& P = m->tc->prec[0];
  TcTables* tab = nullptr;
  FCGNO_TRY(ensure_tables(m, false, g, tab, st));
  TcActs& T = *op->tc_acts;
  TcTrainBufs& tb = T.train;
  BlobLayout BL = blob_layout(d);
  const int lift_blocks = (op->N / kLiftCols) * (op->N / lift_rows(op->N));
  FCGNO_CUDA_TRY(launch_chained(tc_lift_kernel<C>, dim3(lift_blocks, op->B), dim3(kLiftThreads), 0, st, g, r,
                                (const float*)op->logk32, rms, (const int*)nullptr,
                                (const float*)(m->w32 + BL.lift_w), (const float*)(m->w32 + BL.lift_b), tb.v[0],
                                true));
  FCGNO_LAUNCHED();
  for (int l = 0; l < d.layers; ++l) {
    FCGNO_TRY(launch_ana<C>(g, op, tb.v[l], tab, T.part, st));
    FCGNO_TRY(part_to_cx(g, op, T.part, cx[l], st));
    FCGNO_TRY(launch_mixing<C>(g, op, T.part, P.Rr[l], T.chat, st));
    const bool act = l < d.layers - 1;
    FCGNO_TRY(launch_syn_hidden<C>(g, op, tb.v[l], tb.v[l + 1], T.chat, P.W[l], m->w32 + BL.b[l], tab, act,
                                   (act && !tb.recompute) ? tb.h[l] : nullptr, st));
  }
  return FCGNO_OK;
}

fcgno_status tc_train_forward(fcgno_model* m, const fcgno_op* op, const double* r, const double* rms,
                              float* const* cx, cudaStream_t st) {
  if (m->desc.width == 16) return train_forward<16>(m, op, r, rms, cx, st);
  return train_forward<32>(m, op, r, rms, cx, st);
}

fcgno_status tc_train_to_f32(const fcgno_model* m, const fcgno_op* op, int which, float* out, cudaStream_t st) {
  const TcGeom g = make_geom(op->N, m->desc.width, m->desc.modes);
  const TcTrainBufs& tb = op->tc_acts->train;
  const size_t total = (size_t)op->B * op->n * (g.C / 8);
  tc_tile_to_f32_kernel<<<ceil_div(total, 256), 256, 0, st>>>(g, op->B, which < 0 ? tb.gv : tb.v[which], out);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

fcgno_status tc_train_act_bwd(const fcgno_model* m, const fcgno_op* op, int l, const float* gv32, float* gh32,
                              cudaStream_t st) {
  const TcGeom g = make_geom(op->N, m->desc.width, m->desc.modes);
  TcTrainBufs& tb = op->tc_acts->train;
  const size_t total = (size_t)op->B * op->n * (g.C / 8);
  tc_act_bwd_kernel<<<ceil_div(total, 256), 256, 0, st>>>(g, op->B, gv32, tb.gv,
                                                          l < m->desc.layers - 1 ? tb.h[tb.recompute ? 0 : l] : nullptr,
                                                          gh32, tb.gh);
  FCGNO_LAUNCHED();
  return FCGNO_OK;
}

// Activation checkpointing of the BF16 step: layer l's pre-activation rebuilt from its kept
// input by the forward's own kernels on the same inputs (analysis, mixing, synthesis), so the
// values are bit-identical; the synthesis rewrites v[l + 1] with the same bytes.
template <int C>
static fcgno_status train_recompute_layer(fcgno_model* m, const fcgno_op* op, int l, cudaStream_t st) {
  const fcgno_model_desc& d = m->desc;
  const TcGeom g = make_geom(op->N, C, d.modes);
  TcPrecision& P = m->tc->prec[0];
  TcTables* tab = nullptr;
  FCGNO_TRY(ensure_tables(m, false, g, tab, st));
  TcActs& T = *op->tc_acts;
  TcTrainBufs& tb = T.train;
  BlobLayout BL = blob_layout(d);
  FCGNO_TRY(launch_ana<C>(g, op, tb.v[l], tab, T.part, st));
  FCGNO_TRY(launch_mixing<C>(g, op, T.part, P.Rr[l], T.chat, st));
  return launch_syn_hidden<C>(g, op, tb.v[l], tb.v[l + 1], T.chat, P.W[l], m->w32 + BL.b[l], tab, 1, tb.h[0], st);
}

fcgno_status tc_train_recompute_layer(fcgno_model* m, const fcgno_op* op, int l, cudaStream_t st) {
  if (!op->tc_acts->train.recompute || l >= m->desc.layers - 1) return FCGNO_OK;
  if (m->desc.width == 16) return train_recompute_layer<16>(m, op, l, st);
  return train_recompute_layer<32>(m, op, l, st);
}

template <int C>
static fcgno_status train_layer_bwd(fcgno_model* m, const fcgno_op* op, int l, cudaStream_t st) {
  const TcGeom g = make_geom(op->N, C, m->desc.modes);
  TcPrecision& P = m->tc->prec[0];
  TcTables* adj = nullptr;
  FCGNO_TRY(ensure_tables(m, false, g, adj, st, true));
  TcActs& T = *op->tc_acts;
  TcTrainBufs& tb = T.train;
  FCGNO_TRY(launch_ana<C>(g, op, tb.gh, adj, tb.partb, st));
  FCGNO_TRY(part_to_cx(g, op, tb.partb, tb.gspec, st));
  FCGNO_TRY(launch_mixing<C>(g, op, tb.partb, P.RrT[l], T.chat, st));
  // (the adjoint tables' stage-1 table H is the forward's: the p-direction twiddles of e^{+i theta})
  return launch_syn_hidden<C>(g, op, tb.gh, tb.gv, T.chat, P.WT[l], tb.zero, adj, 0, nullptr, st);
}

fcgno_status tc_train_layer_bwd(fcgno_model* m, const fcgno_op* op, int l, cudaStream_t st) {
  if (m->desc.width == 16) return train_layer_bwd<16>(m, op, l, st);
  return train_layer_bwd<32>(m, op, l, st);
}

const float* tc_train_gspec(const fcgno_op* op) { return op->tc_acts->train.gspec; }

}  // namespace fcgno
