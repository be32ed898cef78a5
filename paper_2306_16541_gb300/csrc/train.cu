// train.cu -- training step: forward with saved per-ray state, the
// hand-written backward and Adam.
#include "field.cuh"
#include "render.cuh"

using namespace nr;

extern "C" nr_status nr_train_step(nr_subject *s, const nr_train_batch *b, float *loss_out, void *stream) {
  (void)s; (void)b; (void)loss_out; (void)stream;
  set_error("nr_train_step is not implemented yet");
  return NR_EUNSUPPORTED;
}
