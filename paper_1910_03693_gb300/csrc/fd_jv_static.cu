// Finite-difference Jacobian-vector product whose three work vectors live in a
// statically reserved device array, so that the call itself allocates no
// memory.  Meant for callers that cannot call cudaMalloc once their set-up is
// done: processes whose device memory is already fully reserved by another
// allocator (e.g. a framework's caching allocator), where a new allocation
// would fail, and loops that must not call the allocator at all, because
// cudaFree synchronises the whole device and an allocation can stall behind
// other work.  The residual launches it makes allocate nothing either: the
// work table of the multi-bucket launch is built when the layout or the
// tuning changes.
//
// The reserved array holds three vectors of at most kStaticFdMaxDof doubles
// (6 MiB on every device that loads the library, kept until the process
// exits): R(q), q + eps v and R(q + eps v).  Every call writes each of them
// before reading it, so nothing has to be cleared between calls; the array
// keeps the last call's contents.  All calls share the array: two calls whose
// work overlaps on the GPU (different streams or threads on the same device)
// race on it.  The device address is looked up on the first call on each
// device and cached per device, which is right for the runtime's primary
// context, the only one supported.
#include <mutex>

#include "fr_launch.h"

namespace frgb {

constexpr int64_t kStaticFdMaxDof = 262144;
constexpr int kStaticFdMaxDevices = 64;

static __device__ __align__(256) double g_fd_scratch[3 * kStaticFdMaxDof];

__global__ void k_fd_static_shift(const double* __restrict__ q, double eps, const double* __restrict__ v,
                                  double* __restrict__ qp, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    qp[i] = q[i] + eps * v[i];
}

__global__ void k_fd_static_quotient(const double* __restrict__ R1, const double* __restrict__ R0, double inv_eps,
                                     double* __restrict__ Jv, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Jv[i] = (R1[i] - R0[i]) * inv_eps;
}

// Device address of g_fd_scratch on the current device.  The host-side name of
// the array is only a stand-in, so the address is looked up once per device
// (with that device current) and kept.
static fr_status static_scratch(double** out) {
  static std::mutex mtx;
  static double* addr[kStaticFdMaxDevices] = {};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(e, "fr_jvp_fd_static: cudaGetDevice");
  if (dev < 0 || dev >= kStaticFdMaxDevices) {
    set_error("fr_jvp_fd_static: device index beyond the supported range");
    return FR_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(mtx);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fd_scratch);
    if (e != cudaSuccess) return cuda_check(e, "fr_jvp_fd_static: cudaGetSymbolAddress");
    addr[dev] = static_cast<double*>(p);
  }
  *out = addr[dev];
  return FR_OK;
}

}  // namespace frgb

using namespace frgb;

extern "C" fr_status fr_jvp_fd_static(fr_ctx* c, const double* q_dev, const double* v_dev, double* Jv_dev,
                                      double eps, void* stream) {
  if (!c || !q_dev || !v_dev || !Jv_dev || !(eps > 0.0)) {
    set_error("fr_jvp_fd_static: null pointer or eps <= 0");
    return FR_ERR_INVALID;
  }
  const int64_t n = c->n_dof;
  if (n > kStaticFdMaxDof) {
    set_error("fr_jvp_fd_static: n_dof exceeds the reserved scratch (262144 DOF); use fr_jvp");
    return FR_ERR_INVALID;
  }
  int dev = -1;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return cuda_check(ce, "fr_jvp_fd_static: cudaGetDevice");
  if (dev != c->device) {
    set_error("fr_jvp_fd_static: the current device is not the context's device");
    return FR_ERR_INVALID;
  }
  double* base = nullptr;
  fr_status st = static_scratch(&base);
  if (st != FR_OK) return st;
  double* R0 = base;
  double* qp = base + kStaticFdMaxDof;
  double* R1 = base + 2 * kStaticFdMaxDof;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((n + 255) / 256 < 4864 ? (n + 255) / 256 : 4864);
  st = launch_residual(c, q_dev, R0, FR_F64, s);
  if (st != FR_OK) return st;
  FR_LAUNCH_B(c, "vec", s, 24.0 * n, k_fd_static_shift<<<grid, 256, 0, s>>>(q_dev, eps, v_dev, qp, n));
  st = launch_residual(c, qp, R1, FR_F64, s);
  if (st != FR_OK) return st;
  FR_LAUNCH_B(c, "vec", s, 24.0 * n, k_fd_static_quotient<<<grid, 256, 0, s>>>(R1, R0, 1.0 / eps, Jv_dev, n));
  return cuda_check(cudaGetLastError(), "fr_jvp_fd_static");
}
