// Tensor-core jet GEMMs (placeholder until the tcgen05 kernels land).
#include "tc.h"

namespace pinn {

void tc_init(pinn_handle*) {}
bool tc_layer_supported(const pinn_handle*, int, int64_t) { return false; }
int tc_dw_splits(const pinn_handle*, int, int, int64_t) { return 1; }
pinn_status tc_gemm_fwd(pinn_handle*, const void*, const void*, int, int, int64_t, const EpiArgs&, cudaStream_t) {
  return PINN_ERR_UNSUPPORTED;
}
pinn_status tc_gemm_adj(pinn_handle*, const void*, const void*, int, int, int64_t, const EpiArgs&, cudaStream_t) {
  return PINN_ERR_UNSUPPORTED;
}
pinn_status tc_gemm_dw(pinn_handle*, const void*, const void*, int, int, int64_t, int, float*, cudaStream_t) {
  return PINN_ERR_UNSUPPORTED;
}

}  // namespace pinn
