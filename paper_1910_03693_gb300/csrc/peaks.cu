// Measured arithmetic peak of the device: the denominator of the ALU
// rooflines, taken on the GPU that runs the kernels instead of from unit
// counts and a nominal clock.  Independent FMA chains keep every pipe slot
// busy; the result is kept live by a store that never happens.
#include "fr_launch.h"

namespace frgb {

constexpr int kChains = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(T* out, int64_t iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-1.25)) out[0] = s;   // never true: every chain stays in (0, 1)
}

}  // namespace frgb

using namespace frgb;

extern "C" fr_status fr_fma_rate(fr_prec prec, int64_t iters, double* tflops, void* stream) {
  if (!tflops || iters < 1 || (prec != FR_F64 && prec != FR_F32)) {
    set_error("fr_fma_rate: FR_F64 or FR_F32, iters >= 1");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)(sms > 0 ? sms : 1) * 4u;
  void* sink = nullptr;   // a real buffer behind the never-taken store
  fr_status st = cuda_check(cudaMalloc(&sink, 16), "fr_fma_rate: sink");
  if (st != FR_OK) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, s);
    if (prec == FR_F64) k_fma_rate<double><<<grid, 256, 0, s>>>((double*)sink, iters, 0.999999, 1e-7);
    else k_fma_rate<float><<<grid, 256, 0, s>>>((float*)sink, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1, s);
    st = cuda_check(cudaEventSynchronize(e1), "fr_fma_rate");
    if (st != FR_OK) break;
    cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (st != FR_OK) return st;
  const double fmas = (double)grid * 256.0 * (double)iters * kChains;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return FR_OK;
}
