// F64 kernels of the residual, JVP and VJP: 3D with diagonal metrics.
#include "fr_dispatch.cuh"

namespace frgb {
FR_RUN_CFG(run_f64_3d_diag, double, 3, true)
}  // namespace frgb
