// F32 kernels of the residual, JVP and VJP: 3D with diagonal metrics.
#include "fr_dispatch.cuh"

namespace frgb {
FR_RUN_CFG(run_f32_3d_diag, float, 3, true)
}  // namespace frgb
