// F64 kernels of the residual, JVP and VJP: 2D.
#include "fr_dispatch.cuh"

namespace frgb {
FR_RUN_CFG(run_f64_2d, double, 2, false)
}  // namespace frgb
