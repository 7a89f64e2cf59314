// Elementwise vector kernels and the paper's finite-difference Jacobian-vector
// product J v ~ (R(q + eps v) - R(q)) / eps (Sec. 2.3).
#include <algorithm>

#include "fr_launch.h"

namespace frgb {

static unsigned grid_for(int64_t n) {
  // grid-stride loops: a few waves over 152 SMs
  int64_t b = (n + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

double* vec64(fr_ctx* c, int k) {
  if (!c->d_vec64[k]) {
    if (cudaMalloc(&c->d_vec64[k], sizeof(double) * c->n_dof_cap) != cudaSuccess) c->d_vec64[k] = nullptr;
  }
  return c->d_vec64[k];
}

float* vec32(fr_ctx* c, int k) {
  if (!c->d_vec32[k]) {
    if (cudaMalloc(&c->d_vec32[k], sizeof(float) * c->n_dof_cap) != cudaSuccess) c->d_vec32[k] = nullptr;
  }
  return c->d_vec32[k];
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
__global__ void k_add_scaled(const double* __restrict__ x, double a, const double* __restrict__ y,
                             double* __restrict__ z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = x[i] + a * y[i];
}
__global__ void k_diff_scaled(const double* __restrict__ x, const double* __restrict__ y, double a,
                              double* __restrict__ z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = (x[i] - y[i]) * a;
}
__global__ void k_cast_df(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_cast_fd(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

void vaxpby(fr_ctx* c, double a, const double* x, double b, double* y, int64_t n, cudaStream_t s) {
  FR_LAUNCH_B(c, "vec", s, 24.0 * n, k_axpby<<<grid_for(n), 256, 0, s>>>(a, x, b, y, n));
}
void vadd_scaled(fr_ctx* c, const double* x, double a, const double* y, double* z, int64_t n, cudaStream_t s) {
  FR_LAUNCH_B(c, "vec", s, 24.0 * n, k_add_scaled<<<grid_for(n), 256, 0, s>>>(x, a, y, z, n));
}
void vdiff_scaled(fr_ctx* c, const double* x, const double* y, double a, double* z, int64_t n, cudaStream_t s) {
  FR_LAUNCH_B(c, "vec", s, 24.0 * n, k_diff_scaled<<<grid_for(n), 256, 0, s>>>(x, y, a, z, n));
}
void vcast_f64_f32(fr_ctx* c, const double* x, float* y, int64_t n, cudaStream_t s) {
  FR_LAUNCH_B(c, "vec", s, 12.0 * n, k_cast_df<<<grid_for(n), 256, 0, s>>>(x, y, n));
}
void vcast_f32_f64(fr_ctx* c, const float* x, double* y, int64_t n, cudaStream_t s) {
  FR_LAUNCH_B(c, "vec", s, 12.0 * n, k_cast_fd<<<grid_for(n), 256, 0, s>>>(x, y, n));
}

fr_status launch_fd_jv(fr_ctx* c, const double* q, const double* v, double* Jv, double eps,
                       const double* R0, cudaStream_t s) {
  double* qp = vec64(c, 0);
  double* R1 = vec64(c, 1);
  if (!qp || !R1) {
    set_error("fd_jv: scratch allocation failed");
    return FR_ERR_NOMEM;
  }
  const int64_t n = c->n_dof;
  if (!R0) {
    double* r0 = vec64(c, 2);
    if (!r0) return FR_ERR_NOMEM;
    fr_status st = launch_residual(c, q, r0, FR_F64, s);
    if (st != FR_OK) return st;
    R0 = r0;
  }
  vadd_scaled(c, q, eps, v, qp, n, s);
  fr_status st = launch_residual(c, qp, R1, FR_F64, s);
  if (st != FR_OK) return st;
  vdiff_scaled(c, R1, R0, 1.0 / eps, Jv, n, s);
  return cuda_check(cudaGetLastError(), "fd_jv");
}

}  // namespace frgb
