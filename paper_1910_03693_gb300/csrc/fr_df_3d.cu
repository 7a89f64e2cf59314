// Double-float kernels of the residual: 3D.
#include "fr_dispatch.cuh"

namespace frgb {
FR_RUN_RES_DF(run_df_3d, 3, false)
}  // namespace frgb
