// Double-float kernels of the residual: 2D.
#include "fr_dispatch.cuh"

namespace frgb {
FR_RUN_RES_DF(run_df_2d, 2, false)
}  // namespace frgb
