// F64 kernels of the residual, JVP and VJP: 3D.
#include "fr_dispatch.cuh"

namespace frgb {
FR_RUN_CFG(run_f64_3d, double, 3, false)
}  // namespace frgb
