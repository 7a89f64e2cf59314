// FP32 instantiation of the FR residual, exact JVP and VJP.
#include "fr_dispatch.cuh"

namespace frgb {
fr_status run_op_f32(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s) {
  return run_op<float>(c, op, q, v, out, s);
}
}  // namespace frgb
