// Internal launch helpers shared by the translation units of the library.
#pragma once

#include "fr_internal.h"

namespace frgb {

// Device scratch vectors owned by the context, sized n_dof_capacity (slots
// 0-2 finite-difference Jv, 3 Jv, 4-5 GMRES, 6-9 ESDIRK, 10-11 adaptation and
// tuning, 12 staging of host buffers in fr_pack / fr_unpack).
constexpr int kHostStageVec = 12;
fr_status canonical_on_device(const void* p, bool* on_device);
double* vec64(fr_ctx* c, int k);
float* vec32(fr_ctx* c, int k);

// y = a*x + b*y ; z = x + a*y ; elementwise casts; scaled difference.
void vaxpby(fr_ctx* c, double a, const double* x, double b, double* y, int64_t n, cudaStream_t s);
void vadd_scaled(fr_ctx* c, const double* x, double a, const double* y, double* z, int64_t n, cudaStream_t s);
void vdiff_scaled(fr_ctx* c, const double* x, const double* y, double a, double* z, int64_t n, cudaStream_t s);
void vcast_f64_f32(fr_ctx* c, const double* x, float* y, int64_t n, cudaStream_t s);
void vcast_f32_f64(fr_ctx* c, const float* x, double* y, int64_t n, cudaStream_t s);

// op 0: out = R(q); op 1: out = J(q) v (exact); op 2: out = J(q)^T v;
// op 3: traces of q only (prepares op 4); op 4: J(q) v reusing those traces;
// op 5: autotune the launch configuration on q (out: scratch of n_dof);
// op 6: as op 4, writing -J(q) v in FP64 into out.
fr_status run_op_f64(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);
fr_status run_op_f32(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);
// residual only (op 0): FP64 state in, FP64 R out, double-float arithmetic
fr_status run_op_df(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);

// per-configuration entry points behind run_op_f64/f32 (2D; 3D; 3D with
// diagonal metrics, the axis-aligned affine elements)
void run_f64_2d(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);
void run_f64_3d(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);
void run_f64_3d_diag(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);
void run_f32_2d(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);
void run_f32_3d(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);
void run_f32_3d_diag(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s);
void run_df_2d(fr_ctx* c, const void* q, double* R, cudaStream_t s);
void run_df_3d(fr_ctx* c, const void* q, double* R, cudaStream_t s);
void run_df_3d_diag(fr_ctx* c, const void* q, double* R, cudaStream_t s);

fr_status launch_jvp_prepare(fr_ctx* c, const void* q, fr_prec prec, cudaStream_t s);
fr_status launch_jvp_prepared(fr_ctx* c, const void* q, const void* v, void* Jv, fr_prec prec, cudaStream_t s);
// Same, writing w = -J(q) v in FP64 (the Arnoldi vector), in either precision.
fr_status launch_jvp_prepared_neg64(fr_ctx* c, const void* q, const void* v, double* w, fr_prec prec,
                                    cudaStream_t s);

// z = M^-1 (a w + b u) with the element-Jacobi preconditioner (u optional; z may alias w).
// bscale (optional, device): b is multiplied by *bscale on the device; gate
// (optional): the launches return at entry when *gate is set (gate_closed).
fr_status precond_apply(fr_ctx* c, double a, const double* w, double b, const double* u, double* z, cudaStream_t s,
                        const int* gate = nullptr, const double* bscale = nullptr);
// The same on FP32 vectors (the FP32 Krylov basis).
fr_status precond_apply(fr_ctx* c, double a, const float* w, double b, const float* u, float* z, cudaStream_t s,
                        const int* gate = nullptr, const double* bscale = nullptr);

// Jv = (R(q + eps v) - R0) / eps in FP64; R0 = R(q) is computed when null.
fr_status launch_fd_jv(fr_ctx* c, const double* q, const double* v, double* Jv, double eps,
                       const double* R0, cudaStream_t s);

}  // namespace frgb
