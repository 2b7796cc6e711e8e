// Tensor-core (tcgen05) preconditioner path: placeholder until the kernels land.
#include "internal.cuh"

namespace fcgno {

struct TcModel {};

fcgno_status tc_model_sync(fcgno_model*, cudaStream_t) { return FCGNO_OK; }
void tc_model_free(fcgno_model* m) {
  delete m->tc;
  m->tc = nullptr;
}
fcgno_status no_apply_tc(fcgno_model*, const fcgno_op*, const double*, const double*, const int*, double*, bool,
                         cudaStream_t) {
  set_last_error("tensor-core preconditioner not available in this build");
  return FCGNO_EINVAL;
}

}  // namespace fcgno
