// Double-float kernels of the residual: 3D with diagonal metrics.
#include "fr_dispatch.cuh"

namespace frgb {
FR_RUN_RES_DF(run_df_3d_diag, 3, true)
}  // namespace frgb
