// Launch orchestration of the FR residual and exact JVP, canonical <-> state
// layout conversion, and the C-ABI entry points fr_pack, fr_unpack,
// fr_residual and fr_jvp.
#include <algorithm>
#include <cstdio>
#include <string>
#include <cstring>

#include "fr_launch.h"

namespace frgb {

Timing& timing_of(fr_ctx* c);

// FR_F64 -> FP64 kernels; FR_DF -> double-float kernels (residual only);
// FR_F32 -> FP32 kernels; FR_BF16OP -> FP32 kernels
// reading the bfloat16-rounded operator tables (the kernel arguments point at
// them, so a captured graph keeps the tables it was captured with)
static fr_status run_op_prec(fr_ctx* c, int op, const void* q, const void* v, void* out, fr_prec prec,
                             cudaStream_t s) {
  if (prec == FR_F64) return run_op_f64(c, op, q, v, out, s);
  if (prec == FR_DF) return run_op_df(c, op, q, v, out, s);
  c->bf16op = prec == FR_BF16OP;
  const fr_status st = run_op_f32(c, op, q, v, out, s);
  c->bf16op = false;
  return st;
}

fr_status launch_residual(fr_ctx* c, const void* q, void* R, fr_prec prec, cudaStream_t s) {
  return run_op_prec(c, 0, q, nullptr, R, prec, s);
}

fr_status launch_jvp_exact(fr_ctx* c, const void* q, const void* v, void* Jv, fr_prec prec,
                           cudaStream_t s) {
  return run_op_prec(c, 1, q, v, Jv, prec, s);
}

fr_status launch_jvp_prepare(fr_ctx* c, const void* q, fr_prec prec, cudaStream_t s) {
  return run_op_prec(c, 3, q, nullptr, nullptr, prec, s);
}

fr_status launch_jvp_prepared(fr_ctx* c, const void* q, const void* v, void* Jv, fr_prec prec, cudaStream_t s) {
  return run_op_prec(c, 4, q, v, Jv, prec, s);
}

fr_status launch_jvp_prepared_neg64(fr_ctx* c, const void* q, const void* v, double* w, fr_prec prec,
                                    cudaStream_t s) {
  return run_op_prec(c, 6, q, v, w, prec, s);
}

fr_status launch_vjp(fr_ctx* c, const void* q, const void* w, void* JTw, fr_prec prec, cudaStream_t s) {
  return run_op_prec(c, 2, q, w, JTw, prec, s);
}

// One block per element slot; threads walk the element's [v][sp] block.
template <typename T>
__global__ void pack_kernel(const double* __restrict__ canon, T* __restrict__ q,
                            const int64_t* __restrict__ canon_off, const int64_t* __restrict__ state_off,
                            const int8_t* __restrict__ slot_p, int E, int nd, int nv) {
  for (int64_t sidx = blockIdx.x; sidx < E; sidx += gridDim.x) {
    const int P = slot_p[sidx] + 1;
    const int nsp = nd == 2 ? P * P : P * P * P;
    const int64_t co = canon_off[sidx], so = state_off[sidx];
    for (int k = threadIdx.x; k < nsp * nv; k += blockDim.x) {
      const int v = k / nsp, sp = k % nsp;
      q[so + k] = (T)canon[co + (int64_t)sp * nv + v];
    }
  }
}

template <typename T>
__global__ void unpack_kernel(const T* __restrict__ q, double* __restrict__ canon,
                              const int64_t* __restrict__ canon_off, const int64_t* __restrict__ state_off,
                              const int8_t* __restrict__ slot_p, int E, int nd, int nv) {
  for (int64_t sidx = blockIdx.x; sidx < E; sidx += gridDim.x) {
    const int P = slot_p[sidx] + 1;
    const int nsp = nd == 2 ? P * P : P * P * P;
    const int64_t co = canon_off[sidx], so = state_off[sidx];
    for (int k = threadIdx.x; k < nsp * nv; k += blockDim.x) {
      const int sp = k / nv, v = k % nv;
      canon[co + k] = (double)q[so + (int64_t)v * nsp + sp];
    }
  }
}

// Whether a canonical buffer given to fr_pack / fr_unpack is device memory
// (device or managed allocations, read by the kernels in place) or host memory
// (page-locked or pageable, copied through the staging vector).
fr_status canonical_on_device(const void* p, bool* on_device) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    *on_device = false;
    return FR_OK;
  }
  *on_device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  return FR_OK;
}

fr_status launch_pack(fr_ctx* c, const double* canon, void* q, fr_prec prec, bool unpack, cudaStream_t s) {
  const unsigned g = (unsigned)std::min<int64_t>(c->E, 1 << 20);
  if (!unpack) {
    if (prec == FR_F64)
      FR_LAUNCH_B(c, "pack", s, (double)c->n_dof * (8 + (prec == FR_F64 ? 8 : 4)), pack_kernel<double><<<g, 128, 0, s>>>(canon, (double*)q, c->d_canon_off, c->d_state_off, c->d_slot_p, c->E, c->nd, c->nv));
    else
      FR_LAUNCH_B(c, "pack", s, (double)c->n_dof * (8 + (prec == FR_F64 ? 8 : 4)), pack_kernel<float><<<g, 128, 0, s>>>(canon, (float*)q, c->d_canon_off, c->d_state_off, c->d_slot_p, c->E, c->nd, c->nv));
  } else {
    if (prec == FR_F64)
      FR_LAUNCH_B(c, "pack", s, (double)c->n_dof * (8 + (prec == FR_F64 ? 8 : 4)), unpack_kernel<double><<<g, 128, 0, s>>>((const double*)q, const_cast<double*>(canon), c->d_canon_off, c->d_state_off, c->d_slot_p, c->E, c->nd, c->nv));
    else
      FR_LAUNCH_B(c, "pack", s, (double)c->n_dof * (8 + (prec == FR_F64 ? 8 : 4)), unpack_kernel<float><<<g, 128, 0, s>>>((const float*)q, const_cast<double*>(canon), c->d_canon_off, c->d_state_off, c->d_slot_p, c->E, c->nd, c->nv));
  }
  return cuda_check(cudaGetLastError(), "pack kernel launch");
}

}  // namespace frgb

namespace frgb {
Timing& timing_of(fr_ctx* c) { return c->timing; }
}  // namespace frgb

using namespace frgb;

extern "C" {

fr_status fr_timing(fr_ctx* c, int32_t enable) {
  if (!c) return FR_ERR_INVALID;
  cudaDeviceSynchronize();
  c->timing.collect();
  collect_graph_timers(c);
  c->timing.acc.clear();
  c->timing.launches = 0;
  c->timing.on = enable != 0;
  return FR_OK;
}

fr_status fr_timing_select(fr_ctx* c, const char* names) {
  if (!c) return FR_ERR_INVALID;
  cudaDeviceSynchronize();
  c->timing.collect();
  collect_graph_timers(c);
  c->timing.select.clear();
  if (names) {
    std::string cur;
    for (const char* p = names;; ++p) {
      if (*p == ',' || *p == '\0') {
        if (!cur.empty()) c->timing.select.push_back(cur);
        cur.clear();
        if (*p == '\0') break;
      } else if (*p != ' ') {
        cur += *p;
      }
    }
  }
  c->timing.select_gen += 1;
  return FR_OK;
}

fr_status fr_timing_report(fr_ctx* c, char* buf, int64_t len, int64_t* launches) {
  if (!c || !buf || len <= 0) return FR_ERR_INVALID;
  cudaDeviceSynchronize();
  c->timing.collect();
  collect_graph_timers(c);
  std::string out;
  char line[256];
  for (const auto& kv : c->timing.acc) {
    snprintf(line, sizeof(line), "%s %lld %.6f %.0f %.0f\n", kv.first.c_str(), kv.second.count, kv.second.ms,
             kv.second.bytes, kv.second.flops);
    out += line;
  }
  if ((int64_t)out.size() + 1 > len) return FR_ERR_INVALID;
  std::memcpy(buf, out.c_str(), out.size() + 1);
  if (launches) *launches = c->timing.launches;
  return FR_OK;
}

fr_status fr_device_status(fr_ctx* c, int32_t* status, int32_t clear) {
  if (!c || !status) return FR_ERR_INVALID;
  int v = 0;
  fr_status st = cuda_check(cudaDeviceSynchronize(), "fr_device_status");
  if (st != FR_OK) return st;
  st = cuda_check(cudaMemcpy(&v, c->d_status, sizeof(int), cudaMemcpyDeviceToHost), "fr_device_status");
  if (st != FR_OK) return st;
  if (clear) cudaMemset(c->d_status, 0, sizeof(int));
  *status = v;
  return FR_OK;
}

fr_status fr_autotune(fr_ctx* c, const double* q64_dev, void* stream) {
  if (!c || !q64_dev) {
    set_error("fr_autotune: null argument");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* scr64 = vec64(c, 11);
  float* q32 = vec32(c, 0);
  float* scr32 = vec32(c, 1);
  if (!scr64 || !q32 || !scr32) return FR_ERR_NOMEM;
  const bool timing = c->timing.on;
  c->timing.on = false;
  fr_status st = run_op_f64(c, 5, q64_dev, nullptr, scr64, s);
  if (st == FR_OK) {
    vcast_f64_f32(c, q64_dev, q32, c->n_dof, s);
    st = run_op_f32(c, 5, q32, nullptr, scr32, s);
  }
  c->timing.on = timing;
  if (st != FR_OK) return st;
  return cuda_check(cudaStreamSynchronize(s), "fr_autotune");
}

fr_status fr_tuning_get(const fr_ctx* c, int32_t* table, int32_t* flags) {
  if (!c || !table) return FR_ERR_INVALID;
  std::memcpy(table, c->epb_tab, sizeof(c->epb_tab));
  if (flags)
    *flags = (c->multi_launch ? FR_TUNE_MULTI_LAUNCH : 0) | (c->use_graphs ? FR_TUNE_GRAPHS : 0) |
             (c->use_diag ? FR_TUNE_DIAG_METRICS : 0) | (c->use_fused ? FR_TUNE_FUSED_JVP : 0) |
             (c->df_arnoldi ? FR_TUNE_DF_ARNOLDI : 0) | (c->arnoldi_map == 1 ? FR_TUNE_ARNOLDI_RUNS : 0) |
             (c->use_tma ? FR_TUNE_TMA_FACES : 0) | (c->device_gmres ? FR_TUNE_DEVICE_GMRES : 0) |
             (c->f32_basis ? FR_TUNE_F32_BASIS : 0);
  return FR_OK;
}

fr_status fr_tuning_set(fr_ctx* c, const int32_t* table, int32_t flags) {
  if (!c) return FR_ERR_INVALID;
  if (flags & ~(FR_TUNE_MULTI_LAUNCH | FR_TUNE_GRAPHS | FR_TUNE_DIAG_METRICS | FR_TUNE_FUSED_JVP | FR_TUNE_DF_ARNOLDI |
                FR_TUNE_ARNOLDI_RUNS | FR_TUNE_TMA_FACES | FR_TUNE_DEVICE_GMRES |
                FR_TUNE_F32_BASIS)) {
    set_error("fr_tuning_set: unknown flag bits");
    return FR_ERR_INVALID;
  }
  if (table) {
    for (int i = 0; i < 2 * 3 * (kPM + 1); ++i)
      if (table[i] < 0 ||
          table[i] > (i % (kPM + 1) == 0 ? 2
                      : i % (kPM + 1) == 1 ? (i / (kPM + 1) % 3 == 2 ? 4 : 3)
                                           : 256)) {
        set_error("fr_tuning_set: elements per CTA must lie in [0, 256], multi-bucket choices in [0, 2], "
                  "the weight model in [0, 3], the exact JVP's kernels in [0, 4]");
        return FR_ERR_INVALID;
      }
    std::memcpy(c->epb_tab, table, sizeof(c->epb_tab));
  }
  c->multi_launch = (flags & FR_TUNE_MULTI_LAUNCH) != 0;
  c->use_graphs = (flags & FR_TUNE_GRAPHS) != 0;
  c->use_diag = (flags & FR_TUNE_DIAG_METRICS) != 0;
  c->use_fused = (flags & FR_TUNE_FUSED_JVP) != 0;
  c->df_arnoldi = (flags & FR_TUNE_DF_ARNOLDI) != 0;
  c->arnoldi_map = (flags & FR_TUNE_ARNOLDI_RUNS) != 0 ? 1 : 0;
  c->use_tma = (flags & FR_TUNE_TMA_FACES) != 0;
  c->device_gmres = (flags & FR_TUNE_DEVICE_GMRES) != 0;
  c->f32_basis = (flags & FR_TUNE_F32_BASIS) != 0;
  c->diag = c->diag_mesh && c->use_diag;
  clear_work_cache(c);
  return FR_OK;
}

fr_status fr_pack(fr_ctx* c, const double* canon, void* q_dev, fr_prec prec, void* stream) {
  if (!c || !canon || !q_dev || (prec != FR_F64 && prec != FR_F32 && prec != FR_BF16OP)) return FR_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  bool on_device = false;
  fr_status st = canonical_on_device(canon, &on_device);
  if (st != FR_OK) return st;
  if (on_device) return launch_pack(c, canon, q_dev, prec, false, s);
  // host buffer (page-locked or pageable): one copy into the staging vector
  double* stage = vec64(c, kHostStageVec);
  if (!stage) return FR_ERR_NOMEM;
  st = cuda_check(cudaMemcpyAsync(stage, canon, sizeof(double) * c->n_dof, cudaMemcpyHostToDevice, s),
                  "fr_pack: host to device copy");
  if (st != FR_OK) return st;
  return launch_pack(c, stage, q_dev, prec, false, s);
}

fr_status fr_unpack(fr_ctx* c, const void* q_dev, fr_prec prec, double* canon, void* stream) {
  if (!c || !canon || !q_dev || (prec != FR_F64 && prec != FR_F32 && prec != FR_BF16OP)) return FR_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  bool on_device = false;
  fr_status st = canonical_on_device(canon, &on_device);
  if (st != FR_OK) return st;
  if (on_device) return launch_pack(c, canon, const_cast<void*>(q_dev), prec, true, s);
  double* stage = vec64(c, kHostStageVec);
  if (!stage) return FR_ERR_NOMEM;
  st = launch_pack(c, stage, const_cast<void*>(q_dev), prec, true, s);
  if (st != FR_OK) return st;
  return cuda_check(cudaMemcpyAsync(canon, stage, sizeof(double) * c->n_dof, cudaMemcpyDeviceToHost, s),
                    "fr_unpack: device to host copy");
}

fr_status fr_residual(fr_ctx* c, const void* q_dev, void* R_dev, fr_prec prec, void* stream) {
  if (!c || !q_dev || !R_dev || (prec != FR_F64 && prec != FR_F32 && prec != FR_BF16OP && prec != FR_DF)) {
    set_error("fr_residual: bad argument");
    return FR_ERR_INVALID;
  }
  return launch_residual(c, q_dev, R_dev, prec, (cudaStream_t)stream);
}

fr_status fr_vjp(fr_ctx* c, const void* q_dev, const void* w_dev, void* JTw_dev, fr_prec prec,
                 void* stream) {
  if (!c || !q_dev || !w_dev || !JTw_dev || (prec != FR_F64 && prec != FR_F32 && prec != FR_BF16OP)) {
    set_error("fr_vjp: bad argument");
    return FR_ERR_INVALID;
  }
  return launch_vjp(c, q_dev, w_dev, JTw_dev, prec, (cudaStream_t)stream);
}

fr_status fr_jvp(fr_ctx* c, const void* q_dev, const void* v_dev, void* Jv_dev, fr_prec prec,
                 fr_jv_mode mode, double eps, void* stream) {
  if (!c || !q_dev || !v_dev || !Jv_dev || (prec != FR_F64 && prec != FR_F32 && prec != FR_BF16OP)) {
    set_error("fr_jvp: bad argument");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (mode == FR_JV_EXACT) return launch_jvp_exact(c, q_dev, v_dev, Jv_dev, prec, s);
  if (mode != FR_JV_FD || prec != FR_F64 || !(eps > 0.0)) {
    set_error("fr_jvp: the finite-difference mode is FP64 with eps > 0");
    return FR_ERR_INVALID;
  }
  return launch_fd_jv(c, (const double*)q_dev, (const double*)v_dev, (double*)Jv_dev, eps, nullptr, s);
}

}  // extern "C"
