// Templated launch helpers of the FR residual, JVP and VJP, instantiated once
// per floating-point type in fr_f64.cu and fr_f32.cu.
#pragma once

#include <type_traits>

#include "fr_kernels.cuh"
#include "fr_launch.h"
#include "vjp_kernels.cuh"

namespace frgb {

static inline int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

template <typename T>
inline BasisTab<T>* basis_ptr(fr_ctx* c) {
  return std::is_same<T, double>::value ? (BasisTab<T>*)c->d_basis64 : (BasisTab<T>*)c->d_basis32;
}
template <typename T>
inline MortarTab<T>* mortar_ptr(fr_ctx* c, int Pm, int Ps) {
  return std::is_same<T, double>::value ? (MortarTab<T>*)(c->d_mortar64 + Pm * (kPM + 1) + Ps)
                                        : (MortarTab<T>*)(c->d_mortar32 + Pm * (kPM + 1) + Ps);
}

template <typename T>
inline GeoView<T> geo_view(fr_ctx* c, int p) {
  GeoView<T> g{};
  const int nd = c->nd, NK = nd * nd + 1, P = p + 1;
  const int NSP = ipow(P, nd), NFP = ipow(P, nd - 1);
  const T* aff = std::is_same<T, double>::value ? (const T*)c->d_gaff64 : (const T*)c->d_gaff32;
  if (c->affine) {
    g.vol = aff;
    g.ves = NK;
    g.vks = 1;
    g.vps = 0;
    g.face = aff;
    g.fes = NK;
    g.ffs = 0;
    g.fks = 1;
    g.fps = 0;
  } else {
    g.vol = std::is_same<T, double>::value ? (const T*)c->d_gvol64[p] : (const T*)c->d_gvol32[p];
    g.ves = (int64_t)NK * NSP;
    g.vks = NSP;
    g.vps = 1;
    g.face = std::is_same<T, double>::value ? (const T*)c->d_gface64[p] : (const T*)c->d_gface32[p];
    g.fes = (int64_t)c->nf * NK * NFP;
    g.ffs = NK * NFP;
    g.fks = NFP;
    g.fps = 1;
  }
  return g;
}

static inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------
// dispatch helpers
// ---------------------------------------------------------------------------
template <typename T, int ND, int P, bool VISC>
static void launch_trace_p(const TraceArgs<T>& a, cudaStream_t s) {
  using Cfg = VolCfg<ND, P>;
  constexpr int NV = ND + 2, NF = 2 * ND;
  const size_t smem = (size_t)Cfg::EPB * (NV * Cfg::NSP + NF * NV * Shape<ND, P>::NFP) * sizeof(T);
  auto kern = trace_kernel<T, ND, P, VISC>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  kern<<<nblocks(a.count, Cfg::EPB), Cfg::THREADS, smem, s>>>(a);
}

template <typename T, int ND, bool VISC>
static void launch_trace(fr_ctx* c, const Bucket& b, const T* q, T* trace, cudaStream_t s) {
  TraceArgs<T> a;
  a.q = q;
  a.trace = trace;
  a.slot_elem = c->d_slot_elem;
  a.basis = basis_ptr<T>(c);
  a.geo = geo_view<T>(c, b.p);
  a.state_base = b.state_base;
  a.trace_base = b.trace_base;
  a.count = b.count;
  a.slot_begin = b.slot_begin;
  a.nvt = c->nvt;
  const int P = b.p + 1;
  const double nb = (double)b.count * (ND + 2) * ipow(P, ND) * sizeof(T);
  const double nfl = (double)b.count * 2 * ND * ipow(P, ND - 1) * flops_trace(ND, P, VISC);
  FR_LAUNCH_BF(c, sizeof(T) == 8 ? "trace_f64" : "trace_f32", s, nb, nfl, {
    switch (P) {
      case 2: launch_trace_p<T, ND, 2, VISC>(a, s); break;
      case 3: launch_trace_p<T, ND, 3, VISC>(a, s); break;
      case 4: launch_trace_p<T, ND, 4, VISC>(a, s); break;
      case 5: launch_trace_p<T, ND, 5, VISC>(a, s); break;
      case 6: launch_trace_p<T, ND, 6, VISC>(a, s); break;
    }
  });
}

template <typename T, int ND, int P, bool VISC, int MODE>
static void launch_vol_p(fr_ctx* c, const VolArgs<T>& a, cudaStream_t s) {
  using Cfg = VolCfg<ND, P>;
  using S = typename std::conditional<MODE == 1, Dual<T>, T>::type;
  const size_t smem = (size_t)Cfg::EPB * (ND + 2) * (1 + ND) * Cfg::NSP * sizeof(S);
  auto kern = vol_kernel<T, ND, P, VISC, MODE>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  const unsigned g = nblocks(a.count, Cfg::EPB);
  const char* name = MODE == 1 ? (sizeof(T) == 8 ? "vol_jvp_f64" : "vol_jvp_f32")
                               : (sizeof(T) == 8 ? "vol_res_f64" : "vol_res_f32");
  const double nb = (double)a.count * (ND + 2) * Cfg::NSP * sizeof(T) * (MODE == 1 ? 3 : 2);
  const double nfl = MODE == 1 ? 0.0 : (double)a.count * Cfg::NSP * flops_volume(ND, P, VISC);
  FR_LAUNCH_BF(c, name, s, nb, nfl, kern<<<g, Cfg::THREADS, smem, s>>>(a));
}

template <typename T, int ND, bool VISC, int MODE>
static void launch_vol(fr_ctx* c, const Bucket& b, const T* q, const T* v, T* out, cudaStream_t s) {
  VolArgs<T> a;
  a.q = q;
  a.v = v;
  a.out = out;
  a.fout = (const T*)c->d_fout;
  a.slot_elem = c->d_slot_elem;
  a.basis = basis_ptr<T>(c);
  a.geo = geo_view<T>(c, b.p);
  a.gamma = (T)c->phys.gamma;
  a.mu = (T)c->phys.mu;
  a.kappa = (T)c->phys.kappa;
  a.state_base = b.state_base;
  a.out_base = b.out_base;
  a.count = b.count;
  a.slot_begin = b.slot_begin;
  switch (b.p + 1) {
    case 2: launch_vol_p<T, ND, 2, VISC, MODE>(c, a, s); break;
    case 3: launch_vol_p<T, ND, 3, VISC, MODE>(c, a, s); break;
    case 4: launch_vol_p<T, ND, 4, VISC, MODE>(c, a, s); break;
    case 5: launch_vol_p<T, ND, 5, VISC, MODE>(c, a, s); break;
    case 6: launch_vol_p<T, ND, 6, VISC, MODE>(c, a, s); break;
  }
}

template <typename T, int ND, bool VISC, int MODE>
static void launch_faces(fr_ctx* c, const T* trq, const T* trv, cudaStream_t s) {
  for (const auto& g : c->fgroups) {
    FaceArgs<T> a;
    a.recs = g.d_recs;
    a.trq = trq;
    a.trv = trv;
    a.fout = (T*)c->d_fout;
    a.scratch = (T*)c->d_scratch;
    a.basis = basis_ptr<T>(c);
    a.mortar = g.pm != g.ps ? mortar_ptr<T>(c, g.pm + 1, g.ps + 1) : nullptr;
    a.geo_m = geo_view<T>(c, g.pm);
    a.geo_s = geo_view<T>(c, g.ps);
    a.gamma = (T)c->phys.gamma;
    a.mu = (T)c->phys.mu;
    a.kappa = (T)c->phys.kappa;
    a.n = g.n;
    a.Pm = g.pm + 1;
    a.Ps = g.ps + 1;
    a.nvt = c->nvt;
    a.scratch_base = g.scratch_base;
    const int64_t nm = (int64_t)g.n * ipow(a.Pm, ND - 1);
    FR_LAUNCH_BF(c, MODE == 1 ? (sizeof(T) == 8 ? "face_jvp_f64" : "face_jvp_f32")
                              : (sizeof(T) == 8 ? "face_res_f64" : "face_res_f32"),
                 s, 0.0, MODE == 1 ? 0.0 : (double)nm * flops_face(ND, VISC),
                 face_kernel<T, ND, VISC, MODE><<<nblocks(nm, 128), 128, 0, s>>>(a));
    if (g.pm != g.ps) {
      const int64_t ns = (int64_t)g.n * ipow(a.Ps, ND - 1);
      FR_LAUNCH(c, "mortar_project", s,
                mortar_project_kernel<T, ND, VISC, MODE><<<nblocks(ns, 128), 128, 0, s>>>(a));
    }
  }
  for (const auto& g : c->bgroups) {
    BndArgs<T> a;
    a.recs = g.d_recs;
    a.trq = trq;
    a.trv = trv;
    a.fout = (T*)c->d_fout;
    a.basis = basis_ptr<T>(c);
    a.geo = geo_view<T>(c, g.p);
    a.gamma = (T)c->phys.gamma;
    a.mu = (T)c->phys.mu;
    a.kappa = (T)c->phys.kappa;
    for (int v = 0; v < 5; ++v) a.qinf[v] = (T)c->phys.q_inf[v];
    a.n = g.n;
    a.P = g.p + 1;
    a.kind = g.kind;
    const int64_t nm = (int64_t)g.n * ipow(a.P, ND - 1);
    FR_LAUNCH(c, "boundary", s, bnd_kernel<T, ND, VISC, MODE><<<nblocks(nm, 128), 128, 0, s>>>(a));
  }
}

template <typename T, int ND, bool VISC>
static void residual_impl(fr_ctx* c, const T* q, T* R, cudaStream_t s) {
  T* trq = (T*)c->d_trace_q;
  for (const auto& b : c->buckets) launch_trace<T, ND, VISC>(c, b, q, trq, s);
  launch_faces<T, ND, VISC, 0>(c, trq, nullptr, s);
  for (const auto& b : c->buckets) launch_vol<T, ND, VISC, 0>(c, b, q, nullptr, R, s);
}

// JVP; with q_traces_ready the traces of q in d_trace_q are reused (q is
// fixed during one GMRES solve)
template <typename T, int ND, bool VISC>
static void jvp_impl(fr_ctx* c, const T* q, const T* v, T* Jv, cudaStream_t s, bool q_traces_ready = false) {
  T* trq = (T*)c->d_trace_q;
  T* trv = (T*)c->d_trace_v;
  for (const auto& b : c->buckets) {
    if (!q_traces_ready) launch_trace<T, ND, VISC>(c, b, q, trq, s);
    launch_trace<T, ND, VISC>(c, b, v, trv, s);
  }
  launch_faces<T, ND, VISC, 1>(c, trq, trv, s);
  for (const auto& b : c->buckets) launch_vol<T, ND, VISC, 1>(c, b, q, v, Jv, s);
}


// ---------------------------------------------------------------------------
// VJP: forward traces and face outputs, then volume^T -> face^T -> trace^T
// ---------------------------------------------------------------------------
template <typename T, int ND, int P, bool VISC>
static void launch_vol_adj_p(fr_ctx* c, const VolAdjArgs<T>& a, cudaStream_t s) {
  using Cfg = VolCfg<ND, P>;
  const size_t smem = (size_t)Cfg::EPB * (2 * (ND + 2) + 2 * ND * (ND + 2)) * Cfg::NSP * sizeof(T);
  auto kern = vol_adj_kernel<T, ND, P, VISC>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  FR_LAUNCH_B(c, sizeof(T) == 8 ? "vol_adj_f64" : "vol_adj_f32", s,
              (double)a.count * (ND + 2) * Cfg::NSP * sizeof(T) * 2,
              kern<<<nblocks(a.count, Cfg::EPB), Cfg::THREADS, smem, s>>>(a));
}

template <typename T, int ND, bool VISC>
static void vjp_impl(fr_ctx* c, const T* q, const T* w, T* out, cudaStream_t s) {
  T* trq = (T*)c->d_trace_q;
  T* fbar = (T*)c->d_fbar;
  T* trbar = (T*)c->d_trbar;
  for (const auto& b : c->buckets) launch_trace<T, ND, VISC>(c, b, q, trq, s);
  launch_faces<T, ND, VISC, 0>(c, trq, nullptr, s);
  for (const auto& b : c->buckets) {
    VolAdjArgs<T> a;
    a.q = q;
    a.w = w;
    a.out = out;
    a.fout = (const T*)c->d_fout;
    a.fbar = fbar;
    a.slot_elem = c->d_slot_elem;
    a.basis = basis_ptr<T>(c);
    a.geo = geo_view<T>(c, b.p);
    a.gamma = (T)c->phys.gamma;
    a.mu = (T)c->phys.mu;
    a.kappa = (T)c->phys.kappa;
    a.state_base = b.state_base;
    a.out_base = b.out_base;
    a.count = b.count;
    a.slot_begin = b.slot_begin;
    switch (b.p + 1) {
      case 2: launch_vol_adj_p<T, ND, 2, VISC>(c, a, s); break;
      case 3: launch_vol_adj_p<T, ND, 3, VISC>(c, a, s); break;
      case 4: launch_vol_adj_p<T, ND, 4, VISC>(c, a, s); break;
      case 5: launch_vol_adj_p<T, ND, 5, VISC>(c, a, s); break;
      case 6: launch_vol_adj_p<T, ND, 6, VISC>(c, a, s); break;
    }
  }
  for (const auto& g : c->fgroups) {
    FaceAdjArgs<T> a;
    a.recs = g.d_recs;
    a.trq = trq;
    a.fbar = fbar;
    a.trbar = trbar;
    a.scratch = (T*)c->d_scratch;
    a.basis = basis_ptr<T>(c);
    a.mortar = g.pm != g.ps ? mortar_ptr<T>(c, g.pm + 1, g.ps + 1) : nullptr;
    a.geo_m = geo_view<T>(c, g.pm);
    a.geo_s = geo_view<T>(c, g.ps);
    a.gamma = (T)c->phys.gamma;
    a.mu = (T)c->phys.mu;
    a.kappa = (T)c->phys.kappa;
    a.n = g.n;
    a.Pm = g.pm + 1;
    a.Ps = g.ps + 1;
    a.scratch_base = g.scratch_base;
    const int64_t nm = (int64_t)g.n * ipow(a.Pm, ND - 1);
    FR_LAUNCH(c, "face_adj", s, face_adj_kernel<T, ND, VISC><<<nblocks(nm, 128), 128, 0, s>>>(a));
    if (g.pm != g.ps) {
      const int64_t ns = (int64_t)g.n * ipow(a.Ps, ND - 1);
      FR_LAUNCH(c, "mortar_gather_adj", s,
                mortar_gather_adj_kernel<T, ND, VISC><<<nblocks(ns, 128), 128, 0, s>>>(a));
    }
  }
  for (const auto& g : c->bgroups) {
    BndAdjArgs<T> a;
    a.recs = g.d_recs;
    a.trq = trq;
    a.fbar = fbar;
    a.trbar = trbar;
    a.basis = basis_ptr<T>(c);
    a.geo = geo_view<T>(c, g.p);
    a.gamma = (T)c->phys.gamma;
    a.mu = (T)c->phys.mu;
    a.kappa = (T)c->phys.kappa;
    for (int v = 0; v < 5; ++v) a.qinf[v] = (T)c->phys.q_inf[v];
    a.n = g.n;
    a.P = g.p + 1;
    a.kind = g.kind;
    const int64_t nm = (int64_t)g.n * ipow(a.P, ND - 1);
    FR_LAUNCH(c, "boundary_adj", s, bnd_adj_kernel<T, ND, VISC><<<nblocks(nm, 128), 128, 0, s>>>(a));
  }
  for (const auto& b : c->buckets) {
    TraceAdjArgs<T> a;
    a.trbar = trbar;
    a.out = out;
    a.basis = basis_ptr<T>(c);
    a.state_base = b.state_base;
    a.trace_base = b.trace_base;
    a.count = b.count;
    a.nvt = c->nvt;
    const int P = b.p + 1;
    const int64_t n = (int64_t)b.count * ipow(P, ND);
    const unsigned g = nblocks(n, 256);
    FR_LAUNCH_B(c, "trace_adj", s, (double)n * (ND + 2) * sizeof(T), {
      switch (P) {
        case 2: trace_adj_kernel<T, ND, 2, VISC><<<g, 256, 0, s>>>(a); break;
        case 3: trace_adj_kernel<T, ND, 3, VISC><<<g, 256, 0, s>>>(a); break;
        case 4: trace_adj_kernel<T, ND, 4, VISC><<<g, 256, 0, s>>>(a); break;
        case 5: trace_adj_kernel<T, ND, 5, VISC><<<g, 256, 0, s>>>(a); break;
        case 6: trace_adj_kernel<T, ND, 6, VISC><<<g, 256, 0, s>>>(a); break;
      }
    });
  }
}

template <typename T>
static fr_status run_op(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s) {
  const T* qq = (const T*)q;
  const T* vv = (const T*)v;
  T* oo = (T*)out;
  if (op == 2 && (!c->d_fbar || !c->d_trbar)) {
    if (!c->d_fbar && cudaMalloc(&c->d_fbar, sizeof(double) * c->fout_cap) != cudaSuccess) {
      set_error("fr_vjp: workspace allocation failed");
      return FR_ERR_NOMEM;
    }
    if (!c->d_trbar && cudaMalloc(&c->d_trbar, sizeof(double) * c->trace_cap) != cudaSuccess) {
      set_error("fr_vjp: workspace allocation failed");
      return FR_ERR_NOMEM;
    }
  }
#define FR_OPS(ND, VISC)                                                       \
  if (op == 0) residual_impl<T, ND, VISC>(c, qq, oo, s);                       \
  else if (op == 1) jvp_impl<T, ND, VISC>(c, qq, vv, oo, s);                   \
  else if (op == 2) vjp_impl<T, ND, VISC>(c, qq, vv, oo, s);                   \
  else if (op == 3) { for (const auto& b : c->buckets) launch_trace<T, ND, VISC>(c, b, qq, (T*)c->d_trace_q, s); } \
  else jvp_impl<T, ND, VISC>(c, qq, vv, oo, s, true);
  if (c->nd == 2) {
    if (c->visc) { FR_OPS(2, true) } else { FR_OPS(2, false) }
  } else {
    if (c->visc) { FR_OPS(3, true) } else { FR_OPS(3, false) }
  }
#undef FR_OPS
  return cuda_check(cudaGetLastError(), "FR kernel launch");
}

}  // namespace frgb
