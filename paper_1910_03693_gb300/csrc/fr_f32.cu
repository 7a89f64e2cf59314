// F32 entry of the FR residual, exact JVP and VJP: picks the translation
// unit of the mesh's configuration.
#include "fr_launch.h"

namespace frgb {
fr_status run_op_f32(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s) {
  if (op == 2 && (!c->d_fbar || !c->d_trbar)) {
    if (!c->d_fbar && cudaMalloc(&c->d_fbar, sizeof(double) * c->fout_cap) != cudaSuccess) {
      set_error("fr_vjp: workspace allocation failed");
      return FR_ERR_NOMEM;
    }
    if (!c->d_trbar && cudaMalloc(&c->d_trbar, sizeof(double) * c->trace_cap) != cudaSuccess) {
      set_error("fr_vjp: workspace allocation failed");
      return FR_ERR_NOMEM;
    }
  }
  if (c->nd == 2) run_f32_2d(c, op, q, v, out, s);
  else if (c->diag && op != 2) run_f32_3d_diag(c, op, q, v, out, s);   // the VJP has no diagonal variant
  else run_f32_3d(c, op, q, v, out, s);
  return cuda_check(cudaGetLastError(), "FR kernel launch");
}
}  // namespace frgb
