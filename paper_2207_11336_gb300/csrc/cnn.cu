// Learned residual CNN denoiser (App. C) -- not built yet in this revision.
#include "common.cuh"

namespace pnp {
int cnn_create(pnp_den*, const float*, const int32_t*, int, const int32_t*, int, int, int) {
  return fail(PNP_ERR_UNSUPPORTED, "CNN denoiser not available in this build");
}
void cnn_destroy(pnp_den*) {}
int cnn_denoise(pnp_den*, cudaStream_t, const float*, float*, int, double*, const float*) {
  return fail(PNP_ERR_UNSUPPORTED, "CNN denoiser not available in this build");
}
}  // namespace pnp
