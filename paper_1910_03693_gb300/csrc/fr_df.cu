// Double-float entry of the FR residual: FP64 state in (converted on load by
// the trace and volume kernels), FP64 residual out, every operation in
// between in double-float arithmetic on the FP32 pipe.
// The double-float copies of the operator and geometry tables are made on the
// device from the FP64 ones the first time they are needed.
#include <algorithm>

#include "dfloat.cuh"
#include "fr_launch.h"

namespace frgb {

__global__ void k_to_dfloat(const double* __restrict__ x, dfloat* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = to_dfloat(x[i]);
}

static unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

static fr_status to_df(const double* src, void** dst, int64_t n, cudaStream_t s) {
  if (n <= 0 || !src) return FR_OK;
  if (!*dst && cudaMalloc(dst, sizeof(dfloat) * n) != cudaSuccess) {
    cudaGetLastError();
    set_error("double-float tables: allocation failed");
    return FR_ERR_NOMEM;
  }
  k_to_dfloat<<<grid_for(n), 256, 0, s>>>(src, (dfloat*)*dst, n);
  return cuda_check(cudaGetLastError(), "double-float table conversion");
}

static int ipow_i(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

static fr_status ensure_df(fr_ctx* c, cudaStream_t s) {
  if (c->df_ready) return FR_OK;
  const int nd = c->nd, E = c->E, nf = c->nf;
  const int64_t per_basis = sizeof(BasisTab<double>) / sizeof(double);
  const int64_t per_mortar = sizeof(MortarTab<double>) / sizeof(double);
  fr_status st;
  if ((st = to_df((const double*)c->d_basis64, &c->d_basis_df, per_basis * (kPM + 1), s)) != FR_OK) return st;
  if ((st = to_df((const double*)c->d_mortar64, &c->d_mortar_df, per_mortar * (kPM + 1) * (kPM + 1), s)) != FR_OK)
    return st;
  if (c->affine) {
    if ((st = to_df(c->d_gaff64, &c->d_gaff_df, (int64_t)E * geo_nk_face(nd), s)) != FR_OK) return st;
  } else {
    for (int p = c->p_min; p <= c->p_max; ++p) {
      const int P = p + 1;
      if ((st = to_df(c->d_gvol64[p], &c->d_gvol_df[p], (int64_t)E * geo_nk_vol(nd) * ipow_i(P, nd), s)) != FR_OK)
        return st;
      if ((st = to_df(c->d_gface64[p], &c->d_gface_df[p], (int64_t)E * nf * geo_nk_face(nd) * ipow_i(P, nd - 1), s)) !=
          FR_OK)
        return st;
    }
  }
  c->df_ready = true;
  return FR_OK;
}

fr_status run_op_df(fr_ctx* c, int op, const void* q, const void*, void* out, cudaStream_t s) {
  if (op != 0) {
    set_error("FR_DF evaluates the residual only");
    return FR_ERR_INVALID;
  }
  const fr_status st = ensure_df(c, s);
  if (st != FR_OK) return st;
  // the kernels read the FP64 state and convert it on load
  if (c->nd == 2) run_df_2d(c, q, (double*)out, s);
  else if (c->diag) run_df_3d_diag(c, q, (double*)out, s);
  else run_df_3d(c, q, (double*)out, s);
  return cuda_check(cudaGetLastError(), "FR kernel launch");
}

}  // namespace frgb

// One double-float operation elementwise on FP64 operands (converted to
// double-float first) with the FP64 value of the result: the arithmetic the
// FR_DF residual is built from, exposed so that it can be checked against
// exact rational results.
__global__ void k_df_eval(int op, const double* a, const double* b, const double* c, double* out, int64_t n) {
  using namespace frgb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const dfloat x = to_dfloat(a[i]);
    const dfloat y = b ? to_dfloat(b[i]) : dfloat(0);
    const dfloat z = c ? to_dfloat(c[i]) : dfloat(0);
    dfloat r(0);
    switch (op) {
      case 0: r = x + y; break;
      case 1: r = x - y; break;
      case 2: r = x * y; break;
      case 3: r = dfma(x, y, z); break;
      case 4: r = x / y; break;
      case 5: r = dsqrt(x); break;
      default: r = x; break;
    }
    out[i] = to_double(r);
  }
}

using namespace frgb;

extern "C" fr_status fr_dfloat_eval(int32_t op, const double* a, const double* b, const double* c, double* out,
                                    int64_t n, void* stream) {
  const bool need_b = op >= 0 && op <= 4, need_c = op == 3;
  if (op < 0 || op > 5 || n < 0 || !a || !out || (need_b && !b) || (need_c && !c)) {
    set_error("fr_dfloat_eval: bad argument");
    return FR_ERR_INVALID;
  }
  if (n == 0) return FR_OK;
  k_df_eval<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(op, a, need_b ? b : nullptr, need_c ? c : nullptr, out, n);
  return cuda_check(cudaGetLastError(), "fr_dfloat_eval");
}
