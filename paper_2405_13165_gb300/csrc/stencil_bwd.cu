// stencil_bwd.cu -- adjoint of the GFDM stencil build with respect to the
// particle positions (recomputing moments and factors per particle).
#include "internal.cuh"

namespace mafp {

int build_stencils_backward(mafp_ctx *ctx, int64_t, int32_t, const void *, const uint8_t *,
                            const void *, const int64_t *, const int32_t *, const void *,
                            const void *, void *, cudaStream_t) {
  snprintf(ctx->err, sizeof(ctx->err), "mafp_build_stencils_backward: not built yet");
  return MAFP_ENOTIMPL;
}

}  // namespace mafp
