// mrrr_adjoint.cu -- backward pass (placeholder until the adjoint kernels land).
#include "mrrr_launch.h"

extern "C" {

mrrr_status mrrr_backward(mrrr_plan* plan, int batch, const int64_t* d_off, const double* W, const double* Z,
                          const double* Wbar, const double* Zbar, double tau_rel, int n_max, double* dbar,
                          double* ebar, void* workspace, size_t ws_bytes, mrrr_stream stream) {
  (void)plan; (void)batch; (void)d_off; (void)W; (void)Z; (void)Wbar; (void)Zbar; (void)tau_rel;
  (void)n_max; (void)dbar; (void)ebar; (void)workspace; (void)ws_bytes; (void)stream;
  return MRRR_ERR_NOTIMPL;
}

mrrr_status mrrr_backward_workspace_size(const mrrr_plan* plan, int batch, int n_max, size_t* bytes) {
  if (!plan || !bytes || batch < 0 || n_max < 0) return MRRR_ERR_ARG;
  *bytes = 256;
  return MRRR_OK;
}

}  // extern "C"
