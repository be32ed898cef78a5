// field_tc.cu -- the per-sample field with both MLPs on the tensor cores.
#include "field.cuh"
#include "render.cuh"

namespace nr {

nr_status launch_field_tc(const FieldParams &P, nr_dtype mlp_dtype, int mode, const float4 *in, uint32_t n_fixed,
                          const uint32_t *n_dev, float *out, int device, cudaStream_t st) {
  (void)P; (void)mode; (void)in; (void)n_fixed; (void)n_dev; (void)out; (void)device; (void)st;
  set_error("mlp_dtype %d is not implemented yet", (int)mlp_dtype);
  return NR_EUNSUPPORTED;
}

}  // namespace nr
