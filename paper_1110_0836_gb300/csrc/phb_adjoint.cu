// Reverse-mode adjoint of the fused fit + right-hand side (placeholder until
// the kernel lands; returns PHB_ERR_INVALID_ARG).
#include "phb_internal.cuh"

extern "C" phb_status phb_rhs_adjoint(const phb_plan*, const phb_params*, const double*,
                                      const double*, const double*, const double*, void*, size_t,
                                      double*, double*, int32_t*, phb_stream_t) {
  return PHB_ERR_INVALID_ARG;
}
