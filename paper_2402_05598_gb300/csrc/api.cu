// Handle management and the remaining C-ABI entry points.
#include "internal.cuh"

#include <mutex>
#include <atomic>
#include <string>
#include <vector>

namespace fcgno {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string t_last_error;

void set_last_error(const std::string& msg) { t_last_error = msg; }

// ---- kernel tracing (CUDA events around selected launches)
static std::mutex g_trace_mu;
static std::string g_trace_family;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_trace_events;
static std::vector<cudaEvent_t> g_trace_pool;
static cudaEvent_t g_trace_open = nullptr;
static EventPairs* g_trace_capture = nullptr;
static double g_trace_replay_ms = 0.0;
static uint64_t g_trace_failed = 0;
static std::string g_trace_first_error;

// A failed timing call must not leave a CUDA error behind for the next launch check.
static void trace_note_failure(cudaError_t e) {
  cudaGetLastError();
  if (g_trace_failed++ == 0) g_trace_first_error = cudaGetErrorString(e);
}
static std::atomic<uint64_t> g_trace_gen{0};
static uint64_t g_trace_replay_n = 0;

static cudaEvent_t trace_event() {
  if (!g_trace_pool.empty()) {
    cudaEvent_t e = g_trace_pool.back();
    g_trace_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bool trace_enabled(const char* family) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  return !g_trace_family.empty() && g_trace_family == family;
}
// Inside a stream capture an ordinary event record cannot be timed afterwards; an external
// event-record node re-records the event on every replay like a plain cudaEventRecord.
static cudaError_t trace_record(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  if (cap == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  return cudaEventRecord(e, st);
}
void trace_begin(const char*, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace_open = trace_event();
  const cudaError_t e = trace_record(g_trace_open, st);
  if (e != cudaSuccess) trace_note_failure(e);
}
void trace_end(const char*, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  cudaEvent_t e = trace_event();
  const cudaError_t er = trace_record(e, st);
  if (er != cudaSuccess) trace_note_failure(er);
  if (g_trace_capture)
    g_trace_capture->emplace_back(g_trace_open, e);
  else
    g_trace_events.emplace_back(g_trace_open, e);
  g_trace_open = nullptr;
}
uint64_t trace_generation() { return g_trace_gen.load(); }
void trace_capture_begin(EventPairs* list) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace_capture = list;
}
void trace_capture_end() {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace_capture = nullptr;
}
void trace_accumulate(const EventPairs& pairs) {
  if (pairs.empty()) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  for (auto& pr : pairs) {
    float ms = 0.f;
    const cudaError_t e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e == cudaSuccess) {
      g_trace_replay_ms += ms;
      g_trace_replay_n += 1;
    } else {
      trace_note_failure(e);
    }
  }
}
void trace_release(EventPairs& pairs) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  for (auto& pr : pairs) {
    g_trace_pool.push_back(pr.first);
    g_trace_pool.push_back(pr.second);
  }
  pairs.clear();
}

void solver_ws_free(fcgno_op* op);

BlobLayout blob_layout(const fcgno_model_desc& d) {
  BlobLayout L{};
  const size_t C = d.width, Cp = d.proj_width, M = d.modes, ci = d.in_channels;
  size_t pos = 0;
  L.lift_w = pos;
  pos += C * ci;
  L.lift_b = pos;
  pos += C;
  for (int l = 0; l < d.layers; ++l) {
    L.w[l] = pos;
    pos += C * C;
    L.b[l] = pos;
    pos += C;
    L.r[l] = pos;
    pos += 2 * M * M * C * C * 2;
  }
  L.proj1_w = pos;
  pos += Cp * C;
  L.proj1_b = pos;
  pos += Cp;
  L.proj2_w = pos;
  pos += Cp;
  L.proj2_b = pos;
  pos += 1;
  L.total = pos;
  return L;
}

__global__ void widen_kernel(size_t n, const float* __restrict__ in, double* __restrict__ out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

static bool desc_ok(const fcgno_model_desc* d) {
  return d && d->width >= 1 && d->width <= 64 && d->layers >= 1 && d->layers <= 16 && d->modes >= 1 &&
         d->modes <= 16 && d->proj_width >= 1 && d->proj_width <= 64 && d->in_channels == 2 &&
         (d->output_scale == 0 || d->output_scale == 1);
}

}  // namespace fcgno

using namespace fcgno;

extern "C" size_t fcgno_weight_count(const fcgno_model_desc* desc) {
  if (!desc_ok(desc)) return 0;
  return blob_layout(*desc).total;
}

extern "C" fcgno_status fcgno_model_sync(fcgno_model_t m, void* stream) {
  if (!m) {
    set_last_error("fcgno_model_sync: null model");
    return FCGNO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  widen_kernel<<<ceil_div(m->count, 256), 256, 0, st>>>(m->count, m->w32, m->w64);
  FCGNO_LAUNCHED();
  return tc_model_sync(m, st);
}

extern "C" fcgno_status fcgno_model_set_train_recompute(fcgno_model_t m, int mode) {
  if (!m || mode < 0 || mode > 2) {
    set_last_error("fcgno_model_set_train_recompute: need a model and mode 0 (auto), 1 (always) or 2 (never)");
    return FCGNO_EINVAL;
  }
  m->train_recompute = mode;
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_model_create(const fcgno_model_desc* desc, const float* weights, void* stream,
                                           fcgno_model_t* out) {
  if (!out || !weights || !desc_ok(desc)) {
    set_last_error("fcgno_model_create: need width, proj_width in 1..64, layers in 1..16, modes in 1..16, "
                   "in_channels == 2 and non-null weights/out");
    return FCGNO_EINVAL;
  }
  *out = nullptr;
  fcgno_model* m = new fcgno_model();
  m->desc = *desc;
  m->w32 = weights;
  m->count = blob_layout(*desc).total;
  if (cudaMalloc(&m->w64, m->count * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    set_last_error("fcgno_model_create: out of device memory");
    return FCGNO_ENOMEM;
  }
  fcgno_status rc = fcgno_model_sync(m, stream);
  if (rc != FCGNO_OK) {
    fcgno_model_destroy(m);
    return rc;
  }
  *out = m;
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_model_destroy(fcgno_model_t m) {
  if (!m) return FCGNO_OK;
  no_workspace_free(m);
  tc_model_free(m);
  if (m->w64) cudaFree(m->w64);
  delete m;
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_op_destroy(fcgno_op_t op) {
  if (!op) return FCGNO_OK;
  solver_ws_free(op);
  tc_acts_free(op);
  double* p[] = {op->aE, op->aN, op->diag, op->logk};
  for (double* x : p)
    if (x) cudaFree(x);
  if (op->logk32) cudaFree(op->logk32);
  if (op->kinv) cudaFree(op->kinv);
  delete op;
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_precond_apply(fcgno_model_t model, fcgno_op_t op, const double* r, double* z,
                                            fcgno_prec prec, void* stream) {
  if (!model || !op || !r || !z) {
    set_last_error("fcgno_precond_apply: null argument");
    return FCGNO_EINVAL;
  }
  if (op->N < 2 * model->desc.modes) {
    set_last_error("fcgno_precond_apply: grid smaller than 2*modes");
    return FCGNO_EINVAL;
  }
  if (prec < FCGNO_FP64 || prec > FCGNO_FP32) {
    set_last_error("fcgno_precond_apply: unknown precision");
    return FCGNO_EINVAL;
  }
  if ((prec == FCGNO_BF16 || prec == FCGNO_FP16) && !tc_shape_supported(op->N, model->desc)) {
    set_last_error(std::string("fcgno_precond_apply: ") + tc_shape_rule());
    return FCGNO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // per-instance rms lives in a small scratch owned by the op's solver workspace
  double* rms = nullptr;
  FCGNO_CUDA_TRY(cudaMallocAsync(&rms, sizeof(double) * op->B, st));
  fcgno_status rc = launch_rms(r, op->B, op->n, rms, st);
  if (rc == FCGNO_OK) {
    switch (prec) {
      case FCGNO_FP64:
        rc = no_apply_simt(model, op, r, rms, nullptr, z, true, st);
        break;
      case FCGNO_FP32:
        rc = no_apply_simt(model, op, r, rms, nullptr, z, false, st);
        break;
      case FCGNO_BF16:
      case FCGNO_FP16:
        rc = no_apply_tc(model, op, r, rms, nullptr, z, prec == FCGNO_FP16, st, launch_shape_mode() == 2);
        break;
      default:
        set_last_error("fcgno_precond_apply: unknown precision");
        rc = FCGNO_EINVAL;
    }
  }
  cudaFreeAsync(rms, st);
  return rc;
}

extern "C" fcgno_status fcgno_train_step_loss(fcgno_model_t model, fcgno_op_t op, const double* r, const double* e,
                                              int batch, fcgno_prec prec, int loss_kind, float* loss, float* grad,
                                              void* stream) {
  if (!model || !op || !r || !e || !loss || !grad || batch != op->B) {
    set_last_error("fcgno_train_step: null argument or batch != op batch");
    return FCGNO_EINVAL;
  }
  if (prec != FCGNO_FP32 && prec != FCGNO_FP64 && prec != FCGNO_BF16) {
    set_last_error("fcgno_train_step: precision must be FCGNO_FP32, FCGNO_FP64 or FCGNO_BF16");
    return FCGNO_EINVAL;
  }
  if (prec == FCGNO_BF16 && !tc_shape_supported(op->N, model->desc)) {
    set_last_error(tc_shape_rule());
    return FCGNO_EINVAL;
  }
  if (loss_kind != FCGNO_LOSS_ENERGY && loss_kind != FCGNO_LOSS_L2) {
    set_last_error("fcgno_train_step_loss: loss_kind must be FCGNO_LOSS_ENERGY or FCGNO_LOSS_L2");
    return FCGNO_EINVAL;
  }
  if (op->N < 2 * model->desc.modes) {
    set_last_error("fcgno_train_step: grid smaller than 2*modes");
    return FCGNO_EINVAL;
  }
  return train_step_simt(model, op, r, e, loss, grad, prec, loss_kind == FCGNO_LOSS_L2,
                         (cudaStream_t)stream);
}

extern "C" fcgno_status fcgno_train_step_f64(fcgno_model_t model, fcgno_op_t op, const double* r, const double* e,
                                             int batch, int loss_kind, double* loss, double* grad, void* stream) {
  if (!model || !op || !r || !e || !loss || !grad || batch != op->B) {
    set_last_error("fcgno_train_step_f64: null argument or batch != op batch");
    return FCGNO_EINVAL;
  }
  if (loss_kind != FCGNO_LOSS_ENERGY && loss_kind != FCGNO_LOSS_L2) {
    set_last_error("fcgno_train_step_f64: loss_kind must be FCGNO_LOSS_ENERGY or FCGNO_LOSS_L2");
    return FCGNO_EINVAL;
  }
  if (op->N < 2 * model->desc.modes) {
    set_last_error("fcgno_train_step_f64: grid smaller than 2*modes");
    return FCGNO_EINVAL;
  }
  return train_step_f64(model, op, r, e, loss, grad, loss_kind == FCGNO_LOSS_L2, (cudaStream_t)stream);
}

extern "C" fcgno_status fcgno_train_step(fcgno_model_t model, fcgno_op_t op, const double* r, const double* e,
                                         int batch, fcgno_prec prec, float* loss, float* grad, void* stream) {
  return fcgno_train_step_loss(model, op, r, e, batch, prec, FCGNO_LOSS_ENERGY, loss, grad, stream);
}

extern "C" size_t fcgno_workspace_bytes(int N, int batch, int m_max, const fcgno_model_desc* desc, fcgno_prec prec) {
  if (N < 2 || batch < 1 || m_max < 1) return 0;
  const size_t n = (size_t)N * N;
  size_t bytes = operator_bytes(n, batch) + solver_ws_bytes(n, batch, m_max + 1);
  if (desc_ok(desc)) {
    if (prec == FCGNO_BF16 || prec == FCGNO_FP16)
      bytes += tc_acts_bytes(N, batch, *desc);
    else
      bytes += simt_buffers_bytes(N, batch, *desc, prec == FCGNO_FP64);
  }
  return bytes;
}

extern "C" fcgno_status fcgno_wait_selftest(fcgno_op_t A, double limit_seconds, void* stream) {
  if (!A || !(limit_seconds >= 1e-6 && limit_seconds <= 1.0)) {
    set_last_error("fcgno_wait_selftest: need an operator and 1e-6 <= limit_seconds <= 1");
    return FCGNO_EINVAL;
  }
  return tc_wait_probe(A, (uint64_t)(limit_seconds * 1e9), (cudaStream_t)stream);
}

namespace fcgno {
static std::atomic<int> g_launch_shape{0};
int launch_shape_mode() { return g_launch_shape.load(std::memory_order_relaxed); }
}  // namespace fcgno

extern "C" fcgno_status fcgno_set_launch_shape(int mode) {
  if (mode < 0 || mode > 2) {
    set_last_error("fcgno_set_launch_shape: mode must be 0 (automatic), 1 (wide) or 2 (narrow)");
    return FCGNO_EINVAL;
  }
  g_launch_shape.store(mode, std::memory_order_relaxed);
  return FCGNO_OK;
}

extern "C" int fcgno_precision_supported(int N, const fcgno_model_desc* desc, fcgno_prec prec) {
  if (N < 2 || !desc_ok(desc) || N < 2 * desc->modes) return 0;
  switch (prec) {
    case FCGNO_FP64:
    case FCGNO_FP32:
      return 1;
    case FCGNO_BF16:
    case FCGNO_FP16:
      return tc_shape_supported(N, *desc) ? 1 : 0;
  }
  return 0;
}

extern "C" const char* fcgno_status_str(fcgno_status s) {
  switch (s) {
    case FCGNO_OK: return "ok";
    case FCGNO_EINVAL: return "invalid argument";
    case FCGNO_ENOMEM: return "out of device memory";
    case FCGNO_ECUDA: return "CUDA error";
    case FCGNO_ENOCONV: return "not converged within max_iter";
    case FCGNO_EBREAKDOWN: return "breakdown: (p, A p) zero or not finite";
    case FCGNO_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

extern "C" const char* fcgno_last_error(void) { return t_last_error.c_str(); }

extern "C" uint64_t fcgno_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" fcgno_status fcgno_trace_set(const char* family) {
  std::lock_guard<std::mutex> lk(fcgno::g_trace_mu);
  fcgno::g_trace_family = family ? family : "";
  fcgno::g_trace_gen.fetch_add(1);
  return FCGNO_OK;
}

extern "C" fcgno_status fcgno_trace_collect(double* total_ms, uint64_t* launches) {
  if (!total_ms || !launches) {
    set_last_error("fcgno_trace_collect: null output");
    return FCGNO_EINVAL;
  }
  std::lock_guard<std::mutex> lk(fcgno::g_trace_mu);
  double tot = 0.0;
  for (auto& pr : fcgno::g_trace_events) {
    if (cudaEventSynchronize(pr.second) != cudaSuccess) {
      set_last_error("fcgno_trace_collect: event synchronisation failed");
      return FCGNO_ECUDA;
    }
    float ms = 0.f;
    const cudaError_t e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e == cudaSuccess)
      tot += ms;
    else
      fcgno::trace_note_failure(e);
    fcgno::g_trace_pool.push_back(pr.first);
    fcgno::g_trace_pool.push_back(pr.second);
  }
  if (fcgno::g_trace_failed) {
    set_last_error("fcgno_trace_collect: " + std::to_string(fcgno::g_trace_failed) +
                   " timing calls failed, first: " + fcgno::g_trace_first_error);
    fcgno::g_trace_failed = 0;
  }
  *total_ms = tot + fcgno::g_trace_replay_ms;
  *launches = fcgno::g_trace_events.size() + fcgno::g_trace_replay_n;
  fcgno::g_trace_events.clear();
  fcgno::g_trace_replay_ms = 0.0;
  fcgno::g_trace_replay_n = 0;
  return FCGNO_OK;
}
