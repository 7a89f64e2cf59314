// Templated launch helpers of the FR residual, JVP and VJP, instantiated once
// per floating-point type in fr_f64.cu and fr_f32.cu.
#pragma once

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "fr_kernels.cuh"
#include "fr_launch.h"
#include "fused_jvp.cuh"
#include "vjp_kernels.cuh"

namespace frgb {

static inline int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// Tables of the arithmetic type T: FP64, FP32 (or the bfloat16-rounded FP32
// operators when c->bf16op), double-float (created on first use).
template <typename T>
inline BasisTab<T>* basis_ptr(fr_ctx* c) {
  if (is_dfloat<T>::value) return (BasisTab<T>*)c->d_basis_df;
  return std::is_same<T, double>::value ? (BasisTab<T>*)c->d_basis64
                                        : (BasisTab<T>*)(c->bf16op ? c->d_basis16 : c->d_basis32);
}
template <typename T>
inline MortarTab<T>* mortar_ptr(fr_ctx* c, int Pm, int Ps) {
  if (is_dfloat<T>::value) return (MortarTab<T>*)c->d_mortar_df + Pm * (kPM + 1) + Ps;
  return std::is_same<T, double>::value ? (MortarTab<T>*)(c->d_mortar64 + Pm * (kPM + 1) + Ps)
                                        : (MortarTab<T>*)((c->bf16op ? c->d_mortar16 : c->d_mortar32) + Pm * (kPM + 1) + Ps);
}
template <typename T>
inline const T* typed(const double* a64, const float* a32, const void* adf) {
  if (is_dfloat<T>::value) return (const T*)adf;
  return std::is_same<T, double>::value ? (const T*)a64 : (const T*)a32;
}

// row of the launch-configuration table: FP64 and double-float kernels share
// the FP64 row (same operand size and shared-memory footprint)
template <typename T>
constexpr int prec_row() { return std::is_same<T, float>::value ? 1 : 0; }
template <typename T>
inline const char* kname(const char* f64, const char* f32, const char* df) {
  return is_dfloat<T>::value ? df : (std::is_same<T, double>::value ? f64 : f32);
}

template <typename T>
inline GeoView<T> geo_view(fr_ctx* c, int p) {
  GeoView<T> g{};
  const int nd = c->nd, NKV = geo_nk_vol(nd), NKF = geo_nk_face(nd), P = p + 1;
  const int NSP = ipow(P, nd), NFP = ipow(P, nd - 1);
  const T* aff = typed<T>(c->d_gaff64, c->d_gaff32, c->d_gaff_df);
  if (c->affine) {
    g.vol = aff;
    g.ves = NKF;
    g.vks = 1;
    g.vps = 0;
    g.face = aff;
    g.fes = NKF;
    g.ffs = 0;
    g.fks = 1;
    g.fps = 0;
  } else {
    g.vol = typed<T>(c->d_gvol64[p], c->d_gvol32[p], c->d_gvol_df[p]);
    g.ves = (int64_t)NKV * NSP;
    g.vks = NSP;
    g.vps = 1;
    g.face = typed<T>(c->d_gface64[p], c->d_gface32[p], c->d_gface_df[p]);
    g.fes = (int64_t)c->nf * NKF * NFP;
    g.ffs = NKF * NFP;
    g.fks = NFP;
    g.fps = 1;
  }
  return g;
}

static inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------
// dispatch helpers
// ---------------------------------------------------------------------------
static inline int nsp_of(int nd, int P) { return nd == 2 ? P * P : P * P * P; }

// elements per CTA: tuned value, else as many whole elements as fit 256 threads
static inline int epb_for(fr_ctx* c, int prec, int kind, int P) {
  const int t = c->epb_tab[prec][kind][P];
  const int nsp = nsp_of(c->nd, P);
  const int dflt = nsp >= 256 ? 1 : 256 / nsp;
  return (t > 0 && t * nsp <= 256) ? t : dflt;
}

// Elements per tile of the multi-bucket launch: as many whole elements as fill
// its 256-thread blocks (the tuned per-bucket values size separate launches,
// whose block is e * n_sp threads; a small one here would leave most of the
// block idle).
static inline unsigned sm_count(fr_ctx* c) {
  static int n = 0;   // one device per process here; queried once
  if (n <= 0) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, c->device);
  return n > 0 ? (unsigned)n : 152u;
}

// One launch over all buckets for this precision and kernel kind: the master
// switch, more than one bucket, and the per-kind choice (the autotuner writes
// it into the unused P = 0 slot of the table: 1 yes, 2 no).  Undecided (0):
// one launch while the mesh's solution points fit in 8 full-occupancy waves
// (2048 threads per SM), where launches and tails dominate; beyond that each
// bucket runs alone at its own degree's register footprint (measured: the
// 4M-DOF vortex batch is faster in one launch, the 18M-DOF cylinder and the
// 16M-DOF adapted C-grid per bucket).
static inline bool use_multi(fr_ctx* c, int prec, int kind) {
  if (!c->multi_launch || c->buckets.size() <= 1) return false;
  const int choice = c->epb_tab[prec][kind][0];
  if (choice == 1) return true;
  if (choice == 2) return false;
  return c->n_dof / c->nv <= (int64_t)8 * 2048 * sm_count(c);
}

// Work table of the multi-bucket launch, built when the layout or the tuning
// changed (rebuild_work_table); never allocated here.  Null when it could not
// be built: the caller then launches per bucket.
static const WorkItem* work_items(fr_ctx* c, int prec, int kind, int* n_items) {
  (void)prec;
  (void)kind;
  *n_items = c->n_work;
  return c->n_work > 0 ? c->d_work : nullptr;
}

template <typename KernelT>
static void ensure_smem(KernelT kern, size_t smem, size_t& configured) {
  if (smem > configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
}

template <typename T, int ND, int P, bool VISC, bool DIAG = false>
static void launch_trace_p(const TraceArgs<T>& a, int epb, cudaStream_t s) {
  constexpr int NV = ND + 2, NF = 2 * ND;
  const size_t smem = (size_t)epb * (NV * Shape<ND, P>::NSP + NF * NV * Shape<ND, P>::NFP) * sizeof(T);
  auto kern = trace_kernel<T, ND, P, VISC, DIAG>;
  static size_t configured = 0;
  ensure_smem(kern, smem, configured);
  kern<<<nblocks(a.count, epb), epb * Shape<ND, P>::NSP, smem, s>>>(a, epb);
}

template <typename T, int ND, bool VISC>
static TraceArgs<T> trace_args(fr_ctx* c, const Bucket& b, const T* q, T* trace) {
  TraceArgs<T> a;
  a.gate = c->gate;
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
  return a;
}

// traces of every bucket: one launch per bucket, or one multi-bucket launch
template <typename T, int ND, bool VISC, bool DIAG = false>
static void launch_traces(fr_ctx* c, const T* q, T* trace, cudaStream_t s) {
  const int prec = prec_row<T>();
  double nb = 0.0, nfl = 0.0;
  for (const auto& b : c->buckets) {
    const int P = b.p + 1;
    nb += (double)b.count * values_trace(ND, P, VISC) * sizeof(T);
    nfl += (double)b.count * 2 * ND * ipow(P, ND - 1) * flops_trace(ND, P, VISC, DIAG);
  }
  const char* name = kname<T>("trace_f64", "trace_f32", "trace_df");
  int n_items = 0;
  const WorkItem* items = use_multi(c, prec, 0) ? work_items(c, prec, 0, &n_items) : nullptr;
  if (items) {
    TraceMulti<T> m;
    size_t smem = 0;
    for (size_t i = 0; i < c->buckets.size(); ++i) {
      const Bucket& b = c->buckets[i];
      const int P = b.p + 1, e = epb_multi(ND, P);
      m.b[i] = trace_args<T, ND, VISC>(c, b, q, trace);
      m.P[i] = P;
      m.epb[i] = e;
      smem = std::max(smem, (size_t)e * ((ND + 2) * nsp_of(ND, P) + 2 * ND * (ND + 2) * ipow(P, ND - 1)) * sizeof(T));
    }
    m.items = items;
    m.n_items = n_items;
    auto kern = trace_multi_kernel<T, ND, VISC, DIAG>;
    static size_t configured = 0;
    ensure_smem(kern, smem, configured);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    const unsigned grid = (unsigned)std::max(1, std::min(m.n_items, (int)(std::max(per_sm, 1) * sm_count(c))));
    FR_LAUNCH_BF(c, name, s, nb, nfl, kern<<<grid, 256, smem, s>>>(m));
    return;
  }
  for (const auto& b : c->buckets) {
    const TraceArgs<T> a = trace_args<T, ND, VISC>(c, b, q, trace);
    const int P = b.p + 1, e = epb_for(c, prec, 0, P);
    const double nbb = (double)b.count * values_trace(ND, P, VISC) * sizeof(T);
    const double nfb = (double)b.count * 2 * ND * ipow(P, ND - 1) * flops_trace(ND, P, VISC, DIAG);
    FR_LAUNCH_BF(c, name, s, nbb, nfb, {
      switch (P) {
        case 2: launch_trace_p<T, ND, 2, VISC, DIAG>(a, e, s); break;
        case 3: launch_trace_p<T, ND, 3, VISC, DIAG>(a, e, s); break;
        case 4: launch_trace_p<T, ND, 4, VISC, DIAG>(a, e, s); break;
        case 5: launch_trace_p<T, ND, 5, VISC, DIAG>(a, e, s); break;
        case 6: launch_trace_p<T, ND, 6, VISC, DIAG>(a, e, s); break;
      }
    });
  }
}

template <typename T, int ND, int P, bool VISC, int MODE, bool DIAG = false>
static void launch_vol_p(const VolArgs<T>& a, int epb, cudaStream_t s) {
  using S = typename std::conditional<MODE == 1, Dual<T>, T>::type;
  const size_t smem = (size_t)epb * (ND + 2) * (1 + ND) * Shape<ND, P>::NSP * sizeof(S);
  auto kern = vol_kernel<T, ND, P, VISC, MODE, DIAG>;
  static size_t configured = 0;
  ensure_smem(kern, smem, configured);
  kern<<<nblocks(a.count, epb), epb * Shape<ND, P>::NSP, smem, s>>>(a, epb);
}

template <typename T>
static VolArgs<T> vol_args(fr_ctx* c, const Bucket& b, const T* q, const T* v, T* out, double* out_neg64 = nullptr,
                           double* out64 = nullptr) {
  VolArgs<T> a;
  a.gate = c->gate;
  a.vscale = c->vscale;
  a.q = q;
  a.v = v;
  a.out = out;
  a.out_neg64 = out_neg64;
  a.out64 = out64;
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
  return a;
}

// volume kernel of every bucket: one launch per bucket, or one multi-bucket launch
template <typename T, int ND, bool VISC, int MODE, bool DIAG = false>
static void launch_vols(fr_ctx* c, const T* q, const T* v, T* out, cudaStream_t s, double* out_neg64 = nullptr,
                        double* out64 = nullptr) {
  using S = typename std::conditional<MODE == 1, Dual<T>, T>::type;
  const int prec = prec_row<T>(), kind = MODE == 1 ? 2 : 1;
  const char* name = MODE == 1 ? kname<T>("vol_jvp_f64", "vol_jvp_f32", "vol_jvp_df")
                               : kname<T>("vol_res_f64", "vol_res_f32", "vol_res_df");
  const double out_ratio = (out_neg64 || out64) ? 8.0 / sizeof(T) : 1.0;
  double nb = 0.0, nfl = 0.0;
  for (const auto& b : c->buckets) {
    const int P = b.p + 1;
    nb += (double)b.count * values_volume(ND, P, VISC, MODE == 1, out_ratio) * sizeof(T);
    nfl += MODE == 1 ? 0.0 : (double)b.count * nsp_of(ND, P) * flops_volume(ND, P, VISC, DIAG);
  }
  int n_items = 0;
  const WorkItem* items = use_multi(c, prec, kind) ? work_items(c, prec, kind, &n_items) : nullptr;
  if (items) {
    VolMulti<T> m;
    size_t smem = 0;
    for (size_t i = 0; i < c->buckets.size(); ++i) {
      const Bucket& b = c->buckets[i];
      const int P = b.p + 1, e = epb_multi(ND, P);
      m.b[i] = vol_args<T>(c, b, q, v, out, out_neg64, out64);
      m.P[i] = P;
      m.epb[i] = e;
      smem = std::max(smem, (size_t)e * (ND + 2) * (1 + ND) * nsp_of(ND, P) * sizeof(S));
    }
    m.items = items;
    m.n_items = n_items;
    auto kern = vol_multi_kernel<T, ND, VISC, MODE, DIAG>;
    static size_t configured = 0;
    ensure_smem(kern, smem, configured);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    const unsigned grid = (unsigned)std::max(1, std::min(m.n_items, (int)(std::max(per_sm, 1) * sm_count(c))));
    FR_LAUNCH_BF(c, name, s, nb, nfl, kern<<<grid, 256, smem, s>>>(m));
    return;
  }
  for (const auto& b : c->buckets) {
    const VolArgs<T> a = vol_args<T>(c, b, q, v, out, out_neg64, out64);
    const int P = b.p + 1, e = epb_for(c, prec, kind, P);
    const double nbb = (double)b.count * values_volume(ND, P, VISC, MODE == 1, out_ratio) * sizeof(T);
    const double nfb = MODE == 1 ? 0.0 : (double)b.count * nsp_of(ND, P) * flops_volume(ND, P, VISC, DIAG);
    FR_LAUNCH_BF(c, name, s, nbb, nfb, {
      switch (P) {
        case 2: launch_vol_p<T, ND, 2, VISC, MODE, DIAG>(a, e, s); break;
        case 3: launch_vol_p<T, ND, 3, VISC, MODE, DIAG>(a, e, s); break;
        case 4: launch_vol_p<T, ND, 4, VISC, MODE, DIAG>(a, e, s); break;
        case 5: launch_vol_p<T, ND, 5, VISC, MODE, DIAG>(a, e, s); break;
        case 6: launch_vol_p<T, ND, 6, VISC, MODE, DIAG>(a, e, s); break;
      }
    });
  }
}

template <typename T, int ND, bool VISC, int MODE, bool DIAG = false>
static void launch_faces(fr_ctx* c, const T* trq, const T* trv, cudaStream_t s) {
  for (const auto& g : c->fgroups) {
    FaceArgs<T> a;
    a.gate = c->gate;
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
    a.flux = c->phys.flux;
    a.n = g.n;
    a.Pm = g.pm + 1;
    a.Ps = g.ps + 1;
    a.nvt = c->nvt;
    a.scratch_base = g.scratch_base;
    const int64_t nm = (int64_t)g.n * ipow(a.Pm, ND - 1);
    FR_LAUNCH_BF(c, MODE == 1 ? kname<T>("face_jvp_f64", "face_jvp_f32", "face_jvp_df")
                              : kname<T>("face_res_f64", "face_res_f32", "face_res_df"),
                 s, (double)nm * values_face(ND, VISC, MODE == 1) * sizeof(T),
                 MODE == 1 ? 0.0 : (double)nm * flops_face(ND, VISC, DIAG),
                 face_kernel<T, ND, VISC, MODE, DIAG><<<nblocks(nm, 128), 128, 0, s>>>(a));
    if (g.pm != g.ps) {
      const int64_t ns = (int64_t)g.n * ipow(a.Ps, ND - 1);
      FR_LAUNCH(c, "mortar_project", s,
                mortar_project_kernel<T, ND, VISC, MODE><<<nblocks(ns, 128), 128, 0, s>>>(a));
    }
  }
  for (const auto& g : c->bgroups) {
    BndArgs<T> a;
    a.gate = c->gate;
    a.recs = g.d_recs;
    a.trq = trq;
    a.trv = trv;
    a.fout = (T*)c->d_fout;
    a.basis = basis_ptr<T>(c);
    a.geo = geo_view<T>(c, g.p);
    a.gamma = (T)c->phys.gamma;
    a.mu = (T)c->phys.mu;
    a.kappa = (T)c->phys.kappa;
    a.flux = c->phys.flux;
    for (int v = 0; v < 5; ++v) a.qinf[v] = (T)c->phys.q_inf[v];
    a.n = g.n;
    a.P = g.p + 1;
    a.kind = g.kind;
    const int64_t nm = (int64_t)g.n * ipow(a.P, ND - 1);
    FR_LAUNCH(c, "boundary", s, bnd_kernel<T, ND, VISC, MODE><<<nblocks(nm, 128), 128, 0, s>>>(a));
  }
}

template <typename T, int ND, bool VISC, bool DIAG = false>
static void residual_impl(fr_ctx* c, const T* q, T* R, cudaStream_t s) {
  T* trq = (T*)c->d_trace_q;
  launch_traces<T, ND, VISC, DIAG>(c, q, trq, s);
  launch_faces<T, ND, VISC, 0, DIAG>(c, trq, nullptr, s);
  launch_vols<T, ND, VISC, 0, DIAG>(c, q, nullptr, R, s);
}

// Double-float residual: q is the FP64 state (converted on load), R written
// in FP64 by the volume kernel.
template <typename T, int ND, bool VISC, bool DIAG = false>
static void residual_out64_impl(fr_ctx* c, const T* q, double* R, cudaStream_t s) {
  T* trq = (T*)c->d_trace_q;
  launch_traces<T, ND, VISC, DIAG>(c, q, trq, s);
  launch_faces<T, ND, VISC, 0, DIAG>(c, trq, nullptr, s);
  launch_vols<T, ND, VISC, 0, DIAG>(c, q, nullptr, nullptr, s, nullptr, R);
}

// ---------------------------------------------------------------------------
// Fused JVP (every face interior and conforming): compact traces, then one
// face-and-volume kernel per bucket
// ---------------------------------------------------------------------------
// The fused JVP runs when the mesh allows it, the flag enables it and the
// tuning slot [precision][volume JVP][P = 1] chooses it (1 fused, 2 three
// passes, 0 undecided = three passes): fr_autotune times both and keeps the
// faster (measured on the Taylor-Green box, the fused kernel moves half the
// bytes but is bound by instruction issue and is the slower of the two).
template <typename T>
static inline bool fused_jvp_on(const fr_ctx* c) {
  return c->fused_ok && c->use_fused && c->epb_tab[prec_row<T>()][2][1] == 1;
}
// The compact three-pass JVP (compact traces, the compact face kernel, the
// volume kernel) on the same meshes: slot value 3, and the undecided default.
template <typename T>
static inline bool compact_jvp_on(const fr_ctx* c) {
  const int ch = c->epb_tab[prec_row<T>()][2][1];
  return c->fused_ok && c->use_fused && (ch == 3 || ch == 0 || ch == 4);
}

// The compact passes with the tangent's traces formed in the face kernel
// (slot value 4): FP32 with bulk-copy staging, every face group of a degree
// whose face points lie within one warp and whose blocks are multiples of 16
// bytes, and v's element blocks 16-byte aligned in every bucket (else the
// three compact passes run).
template <typename T, int ND, bool VISC>
static bool cface_vt_usable(const fr_ctx* c, const T* v) {
  if constexpr (!std::is_same<T, float>::value) {
    return false;
  } else {
    if (!c->use_tma) return false;
    for (const auto& g : c->fgroups) {
      bool ok = false;
      switch (g.pm + 1) {
        case 2: ok = CFaceVt<T, ND, 2, VISC>::OK; break;
        case 3: ok = CFaceVt<T, ND, 3, VISC>::OK; break;
        case 4: ok = CFaceVt<T, ND, 4, VISC>::OK; break;
        case 5: ok = CFaceVt<T, ND, 5, VISC>::OK; break;
        case 6: ok = CFaceVt<T, ND, 6, VISC>::OK; break;
      }
      if (!ok) return false;
    }
    for (const auto& b : c->buckets)
      if (reinterpret_cast<uintptr_t>(v + b.state_base) % 16 != 0) return false;
    return true;
  }
}

template <typename T, int ND, int P, bool VISC>
static void launch_ctrace_p(const CTraceArgs<T>& a, int epb, cudaStream_t s) {
  const size_t smem = (size_t)epb * (ND + 2) * Shape<ND, P>::NSP * sizeof(T);
  ctrace_kernel<T, ND, P, VISC><<<nblocks(a.count, epb), epb * Shape<ND, P>::NSP, smem, s>>>(a, epb);
}

template <typename T, int ND, bool VISC>
static void launch_ctraces(fr_ctx* c, const T* q, T* out, cudaStream_t s) {
  constexpr int NV = ND + 2, NF = 2 * ND, CT = VISC ? 2 * NV : NV;
  for (const auto& b : c->buckets) {
    const int P = b.p + 1, e = epb_multi(ND, P);
    CTraceArgs<T> a;
    a.gate = c->gate;
    a.q = q;
    a.out = out;
    a.basis = basis_ptr<T>(c);
    a.state_base = b.state_base;
    a.ctrace_base = b.ctrace_base;
    a.count = b.count;
    const double nb = (double)b.count * (NV * nsp_of(ND, P) + NF * CT * ipow(P, ND - 1)) * sizeof(T);
    FR_LAUNCH_B(c, kname<T>("ctrace_f64", "ctrace_f32", "ctrace_df"), s, nb, {
      switch (P) {
        case 2: launch_ctrace_p<T, ND, 2, VISC>(a, e, s); break;
        case 3: launch_ctrace_p<T, ND, 3, VISC>(a, e, s); break;
        case 4: launch_ctrace_p<T, ND, 4, VISC>(a, e, s); break;
        case 5: launch_ctrace_p<T, ND, 5, VISC>(a, e, s); break;
        case 6: launch_ctrace_p<T, ND, 6, VISC>(a, e, s); break;
      }
    });
  }
}

// Elements per CTA of the fused kernel: as many as fill 256 threads, at most as
// many as leave shared memory for two CTAs on an SM.
template <typename T, int ND, int P, bool VISC>
static int fused_epb() {
  const size_t per = (size_t)FusedSmem<ND, P, VISC>::PER * sizeof(T);
  const int by_smem = (int)std::max<size_t>(1, (size_t)(113 * 1024) / per);
  return std::max(1, std::min(epb_multi(ND, P), by_smem));
}

template <typename T, int ND, int P, bool VISC, bool DIAG>
static void launch_fused_p(const FusedArgs<T>& a, cudaStream_t s) {
  const int epb = fused_epb<T, ND, P, VISC>();
  const size_t smem = (size_t)epb * FusedSmem<ND, P, VISC>::PER * sizeof(T);
  auto kern = fused_jvp_kernel<T, ND, P, VISC, DIAG>;
  static size_t configured = 0;
  ensure_smem(kern, smem, configured);
  kern<<<nblocks(a.count, epb), epb * Shape<ND, P>::NSP, smem, s>>>(a, epb);
}

template <typename T, int ND, bool VISC, bool DIAG>
static void jvp_fused_impl(fr_ctx* c, const T* q, const T* v, T* Jv, cudaStream_t s, bool q_traces_ready,
                           double* neg64) {
  constexpr int NV = ND + 2, NF = 2 * ND, CT = VISC ? 2 * NV : NV;
  T* trq = (T*)c->d_trace_q;
  T* trv = (T*)c->d_trace_v;
  if (!q_traces_ready) launch_ctraces<T, ND, VISC>(c, q, trq, s);
  launch_ctraces<T, ND, VISC>(c, v, trv, s);
  for (const auto& b : c->buckets) {
    FusedArgs<T> a;
    a.gate = c->gate;
    a.vscale = c->vscale;
    a.q = q;
    a.v = v;
    a.trq = trq;
    a.trv = trv;
    a.out = Jv;
    a.out_neg64 = neg64;
    a.nbr = (const FusedNbr*)c->d_fnbr;
    a.slot_elem = c->d_slot_elem;
    a.basis = basis_ptr<T>(c);
    a.geo = geo_view<T>(c, b.p);
    a.gamma = (T)c->phys.gamma;
    a.mu = (T)c->phys.mu;
    a.kappa = (T)c->phys.kappa;
    a.flux = c->phys.flux;
    a.state_base = b.state_base;
    a.ctrace_base = b.ctrace_base;
    a.count = b.count;
    a.slot_begin = b.slot_begin;
    const int P = b.p + 1, NSP = nsp_of(ND, P), NFP = ipow(P, ND - 1);
    // q and v in; the neighbours' compact traces of q and v; J v out (FP64 when negated)
    const double nb = (double)b.count * ((2.0 * NV * NSP + 2.0 * NF * CT * NFP) * sizeof(T) +
                                         (double)NV * NSP * (neg64 ? 8 : sizeof(T)));
    FR_LAUNCH_B(c, kname<T>("fused_jvp_f64", "fused_jvp_f32", "fused_jvp_df"), s, nb, {
      switch (P) {
        case 2: launch_fused_p<T, ND, 2, VISC, DIAG>(a, s); break;
        case 3: launch_fused_p<T, ND, 3, VISC, DIAG>(a, s); break;
        case 4: launch_fused_p<T, ND, 4, VISC, DIAG>(a, s); break;
        case 5: launch_fused_p<T, ND, 5, VISC, DIAG>(a, s); break;
        case 6: launch_fused_p<T, ND, 6, VISC, DIAG>(a, s); break;
      }
    });
  }
}

template <typename T, int ND, int P, bool VISC, bool DIAG>
static void launch_cface_p(fr_ctx* c, const CFaceArgs<T>& a, cudaStream_t s) {
  constexpr int NV = ND + 2;
  constexpr int NFP = ND == 2 ? P : P * P;
  constexpr int FB = NFP >= 128 ? 1 : 128 / NFP;
  constexpr int CT = VISC ? 2 * NV : NV;
  // staged by bulk copies in FP32 where every block is a multiple of 16 bytes
  // and a warp holds the tile's faces (3D p = 1, 3, 5); the two buffers then
  // stay within the 48 KB of static shared memory
  if constexpr (std::is_same<T, float>::value && (CT * NFP * (int)sizeof(T)) % 16 == 0 && FB <= 32 &&
                2 * FB * 4 * CT * NFP * (int)sizeof(T) <= 48 * 1024) {
    if (c->use_tma) {
      const int ntiles = (a.n + FB - 1) / FB;
      const unsigned grid = (unsigned)std::max(1, std::min(ntiles, 4 * (int)sm_count(c)));
      cface_tma_kernel<T, ND, P, VISC, DIAG><<<grid, FB * NFP, 0, s>>>(a, c->d_status);
      return;
    }
  }
  cface_kernel<T, ND, P, VISC, DIAG><<<nblocks(a.n, FB), FB * NFP, 0, s>>>(a);
}

template <typename T, int ND, int P, bool VISC, bool DIAG>
static void launch_cface_vt_p(fr_ctx* c, const CFaceArgs<T>& a, cudaStream_t s) {
  using C = CFaceVt<T, ND, P, VISC>;
  if constexpr (std::is_same<T, float>::value && C::OK) {
    auto kern = cface_vt_kernel<T, ND, P, VISC, DIAG>;
    static size_t configured = 0;
    static int per_sm = 0;
    if (configured == 0)
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    ensure_smem(kern, C::SMEM, configured);
    if (per_sm == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, C::SMEM);
      per_sm = std::max(per_sm, 1);
    }
    const int ntiles = (a.n + C::FB - 1) / C::FB;
    const unsigned grid = (unsigned)std::max(1, std::min(ntiles, per_sm * (int)sm_count(c)));
    kern<<<grid, 128, C::SMEM, s>>>(a, c->d_status);
  }
}

template <typename T, int ND, bool VISC, bool DIAG>
static void jvp_compact_impl(fr_ctx* c, const T* q, const T* v, T* Jv, cudaStream_t s, bool q_traces_ready,
                             double* neg64) {
  constexpr int NV = ND + 2, CT = VISC ? 2 * NV : NV;
  T* trq = (T*)c->d_trace_q;
  T* trv = (T*)c->d_trace_v;
  if (!q_traces_ready) launch_ctraces<T, ND, VISC>(c, q, trq, s);
  const bool vt = c->epb_tab[prec_row<T>()][2][1] == 4 && cface_vt_usable<T, ND, VISC>(c, v);
  if (vt) {
    for (const auto& g : c->fgroups) {
      const Bucket* bk = nullptr;
      for (const auto& b : c->buckets)
        if (b.p == g.pm) bk = &b;
      CFaceArgs<T> a;
      a.gate = c->gate;
      a.recs = g.d_recs;
      a.trq = trq;
      a.fout = (T*)c->d_fout;
      a.basis = basis_ptr<T>(c);
      a.geo = geo_view<T>(c, g.pm);
      a.gamma = (T)c->phys.gamma;
      a.mu = (T)c->phys.mu;
      a.kappa = (T)c->phys.kappa;
      a.flux = c->phys.flux;
      a.n = g.n;
      a.nvt = c->nvt;
      a.v = v;
      a.state_base = bk->state_base;
      a.trace_base = bk->trace_base;
      a.ctrace_base = bk->ctrace_base;
      const int P = g.pm + 1, NFP = ipow(P, ND - 1), NSP = nsp_of(ND, P);
      // both sides' compact traces of q and elements of v in; both sides' face outputs out
      const double nb =
          (double)g.n * (NFP * (2.0 * CT + 2.0 * (VISC ? 3 : 1) * NV) + 2.0 * NV * NSP) * sizeof(T);
      FR_LAUNCH_B(c, kname<T>("cface_vt_jvp_f64", "cface_vt_jvp_f32", "cface_vt_jvp_df"), s, nb, {
        switch (P) {
          case 2: launch_cface_vt_p<T, ND, 2, VISC, DIAG>(c, a, s); break;
          case 3: launch_cface_vt_p<T, ND, 3, VISC, DIAG>(c, a, s); break;
          case 4: launch_cface_vt_p<T, ND, 4, VISC, DIAG>(c, a, s); break;
          case 5: launch_cface_vt_p<T, ND, 5, VISC, DIAG>(c, a, s); break;
          case 6: launch_cface_vt_p<T, ND, 6, VISC, DIAG>(c, a, s); break;
        }
      });
    }
    launch_vols<T, ND, VISC, 1, DIAG>(c, q, v, Jv, s, neg64);
    return;
  }
  launch_ctraces<T, ND, VISC>(c, v, trv, s);
  for (const auto& g : c->fgroups) {
    CFaceArgs<T> a;
    a.gate = c->gate;
    a.recs = g.d_recs;
    a.trq = trq;
    a.trv = trv;
    a.fout = (T*)c->d_fout;
    a.basis = basis_ptr<T>(c);
    a.geo = geo_view<T>(c, g.pm);
    a.gamma = (T)c->phys.gamma;
    a.mu = (T)c->phys.mu;
    a.kappa = (T)c->phys.kappa;
    a.flux = c->phys.flux;
    a.n = g.n;
    a.nvt = c->nvt;
    const int P = g.pm + 1, NFP = ipow(P, ND - 1);
    // both sides' compact traces of q and v in; both sides' face outputs out
    const double nb = (double)g.n * NFP * (4.0 * CT + 2.0 * (VISC ? 3 : 1) * NV) * sizeof(T);
    FR_LAUNCH_B(c, kname<T>("cface_jvp_f64", "cface_jvp_f32", "cface_jvp_df"), s, nb, {
      switch (P) {
        case 2: launch_cface_p<T, ND, 2, VISC, DIAG>(c, a, s); break;
        case 3: launch_cface_p<T, ND, 3, VISC, DIAG>(c, a, s); break;
        case 4: launch_cface_p<T, ND, 4, VISC, DIAG>(c, a, s); break;
        case 5: launch_cface_p<T, ND, 5, VISC, DIAG>(c, a, s); break;
        case 6: launch_cface_p<T, ND, 6, VISC, DIAG>(c, a, s); break;
      }
    });
  }
  launch_vols<T, ND, VISC, 1, DIAG>(c, q, v, Jv, s, neg64);
}

// JVP; with q_traces_ready the traces of q in d_trace_q are reused (q is
// fixed during one GMRES solve)
template <typename T, int ND, bool VISC, bool DIAG = false>
static void jvp_impl(fr_ctx* c, const T* q, const T* v, T* Jv, cudaStream_t s, bool q_traces_ready = false,
                     double* neg64 = nullptr) {
  if constexpr (!is_dfloat<T>::value) {
    if (fused_jvp_on<T>(c)) {
      jvp_fused_impl<T, ND, VISC, DIAG>(c, q, v, Jv, s, q_traces_ready, neg64);
      return;
    }
    if (compact_jvp_on<T>(c)) {
      jvp_compact_impl<T, ND, VISC, DIAG>(c, q, v, Jv, s, q_traces_ready, neg64);
      return;
    }
  }
  T* trq = (T*)c->d_trace_q;
  T* trv = (T*)c->d_trace_v;
  if (!q_traces_ready) launch_traces<T, ND, VISC, DIAG>(c, q, trq, s);
  launch_traces<T, ND, VISC, DIAG>(c, v, trv, s);
  launch_faces<T, ND, VISC, 1, DIAG>(c, trq, trv, s);
  launch_vols<T, ND, VISC, 1, DIAG>(c, q, v, Jv, s, neg64);
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
  launch_traces<T, ND, VISC>(c, q, trq, s);
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
    a.flux = c->phys.flux;
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
    a.flux = c->phys.flux;
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

// ---------------------------------------------------------------------------
// Autotuner: elements per CTA of the trace and volume kernels for every
// degree present, then one launch per bucket vs the multi-bucket launch.
// Candidates are timed with CUDA events (best of `reps`) on the caller's state.
// ---------------------------------------------------------------------------
template <typename F>
static float time_best(int reps, cudaStream_t s, F&& f) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  f();   // warm-up
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, s);
    f();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

template <typename T, int ND, bool VISC, bool DIAG = false>
static void autotune_impl(fr_ctx* c, const T* q, T* scratch, int reps, cudaStream_t s) {
  const int prec = prec_row<T>();
  T* trq = (T*)c->d_trace_q;
  T* trv = (T*)c->d_trace_v;
  const bool multi_saved = c->multi_launch;
  c->multi_launch = false;
  for (int kind = 0; kind < 3; ++kind) {
    // valid face data for the volume kernels
    if (kind == 1) residual_impl<T, ND, VISC, DIAG>(c, q, scratch, s);
    if (kind == 2) jvp_impl<T, ND, VISC, DIAG>(c, q, q, scratch, s);
    for (const auto& b : c->buckets) {
      const int P = b.p + 1, nsp = nsp_of(ND, P);
      std::vector<int> cand;
      for (int e = 1; e * nsp <= 256; e *= 2) cand.push_back(e);
      const int dflt = nsp >= 256 ? 1 : 256 / nsp;
      if (std::find(cand.begin(), cand.end(), dflt) == cand.end()) cand.push_back(dflt);
      float best = 1e30f;
      int best_e = dflt;
      for (int e : cand) {
        float ms = 1e30f;
        if (kind == 0) {
          const TraceArgs<T> a = trace_args<T, ND, VISC>(c, b, q, trq);
          ms = time_best(reps, s, [&] {
            switch (P) {
              case 2: launch_trace_p<T, ND, 2, VISC, DIAG>(a, e, s); break;
              case 3: launch_trace_p<T, ND, 3, VISC, DIAG>(a, e, s); break;
              case 4: launch_trace_p<T, ND, 4, VISC, DIAG>(a, e, s); break;
              case 5: launch_trace_p<T, ND, 5, VISC, DIAG>(a, e, s); break;
              case 6: launch_trace_p<T, ND, 6, VISC, DIAG>(a, e, s); break;
            }
          });
        } else {
          const VolArgs<T> a = vol_args<T>(c, b, q, kind == 2 ? q : nullptr, scratch);
          ms = time_best(reps, s, [&] {
            if (kind == 1) {
              switch (P) {
                case 2: launch_vol_p<T, ND, 2, VISC, 0, DIAG>(a, e, s); break;
                case 3: launch_vol_p<T, ND, 3, VISC, 0, DIAG>(a, e, s); break;
                case 4: launch_vol_p<T, ND, 4, VISC, 0, DIAG>(a, e, s); break;
                case 5: launch_vol_p<T, ND, 5, VISC, 0, DIAG>(a, e, s); break;
                case 6: launch_vol_p<T, ND, 6, VISC, 0, DIAG>(a, e, s); break;
              }
            } else {
              switch (P) {
                case 2: launch_vol_p<T, ND, 2, VISC, 1, DIAG>(a, e, s); break;
                case 3: launch_vol_p<T, ND, 3, VISC, 1, DIAG>(a, e, s); break;
                case 4: launch_vol_p<T, ND, 4, VISC, 1, DIAG>(a, e, s); break;
                case 5: launch_vol_p<T, ND, 5, VISC, 1, DIAG>(a, e, s); break;
                case 6: launch_vol_p<T, ND, 6, VISC, 1, DIAG>(a, e, s); break;
              }
            }
          });
        }
        if (ms < best) {
          best = ms;
          best_e = e;
        }
      }
      c->epb_tab[prec][kind][P] = best_e;
    }
  }
  (void)trv;
  clear_work_cache(c);
  // per kernel kind: one launch per bucket against one multi-bucket launch,
  // with the tuned elements per CTA (the multi kernel carries the register
  // footprint of its largest degree, so large meshes usually prefer separate
  // launches and small batches of buckets the single one)
  c->multi_launch = true;
  if (c->buckets.size() > 1) {
    residual_impl<T, ND, VISC, DIAG>(c, q, scratch, s);
    for (int kind = 0; kind < 3; ++kind) {
      if (kind == 2) jvp_impl<T, ND, VISC, DIAG>(c, q, q, scratch, s);
      float t[2];
      for (int m = 0; m < 2; ++m) {
        c->epb_tab[prec][kind][0] = m == 0 ? 2 : 1;
        t[m] = time_best(reps + 2, s, [&] {
          if (kind == 0) launch_traces<T, ND, VISC, DIAG>(c, q, trq, s);
          else if (kind == 1) launch_vols<T, ND, VISC, 0, DIAG>(c, q, nullptr, scratch, s);
          else launch_vols<T, ND, VISC, 1, DIAG>(c, q, q, scratch, s);
        });
      }
      c->epb_tab[prec][kind][0] = t[1] <= t[0] ? 1 : 2;
    }
  }
  c->multi_launch = multi_saved;
  // keep the tuned table only if the residual plus the JVP beat the default
  // configuration end to end (the per-kernel timings above see each group alone)
  auto both = [&] {
    residual_impl<T, ND, VISC, DIAG>(c, q, scratch, s);
    jvp_impl<T, ND, VISC, DIAG>(c, q, q, scratch, s);
  };
  int tuned[3][kPM + 1];
  std::memcpy(tuned, c->epb_tab[prec], sizeof(tuned));
  clear_work_cache(c);
  const float t_tuned = time_best(reps + 2, s, both);
  std::memset(c->epb_tab[prec], 0, sizeof(tuned));
  for (int k = 0; k < 3; ++k) c->epb_tab[prec][k][1] = tuned[k][1];   // the weight model is not tuned
  clear_work_cache(c);
  const float t_default = time_best(reps + 2, s, both);
  if (t_tuned <= t_default) std::memcpy(c->epb_tab[prec], tuned, sizeof(tuned));
  clear_work_cache(c);
  // fused JVP against the three passes (meshes whose faces are all interior
  // and conforming), with the launch configuration just kept
  if constexpr (!is_dfloat<T>::value) {
    if (c->fused_ok && c->use_fused) {
      float best = 1e30f;
      int choice = 2;
      // 1 fused, 2 trace-gradient three passes, 3 compact three passes, 4 the
      // compact passes with the tangent's traces formed in the face kernel
      for (int m = 1; m <= 4; ++m) {
        if (m == 4 && !cface_vt_usable<T, ND, VISC>(c, q)) continue;
        c->epb_tab[prec][2][1] = m;
        clear_graphs(c);
        const float t = time_best(reps + 2, s, [&] { jvp_impl<T, ND, VISC, DIAG>(c, q, q, scratch, s); });
        if (t < best) {
          best = t;
          choice = m;
        }
      }
      c->epb_tab[prec][2][1] = choice;
      clear_work_cache(c);
    }
  }
}

// One operation for one (dimension, viscosity, metric) configuration.
template <typename T, int ND, bool VISC, bool DIAG>
static void run_op_cfg(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s) {
  const T* qq = (const T*)q;
  const T* vv = (const T*)v;
  T* oo = (T*)out;
  if (op == 0) residual_impl<T, ND, VISC, DIAG>(c, qq, oo, s);
  else if (op == 1) jvp_impl<T, ND, VISC, DIAG>(c, qq, vv, oo, s);
  else if (op == 2) vjp_impl<T, ND, VISC>(c, qq, vv, oo, s);
  else if (op == 3) {
    if (fused_jvp_on<T>(c) || compact_jvp_on<T>(c)) launch_ctraces<T, ND, VISC>(c, qq, (T*)c->d_trace_q, s);
    else launch_traces<T, ND, VISC, DIAG>(c, qq, (T*)c->d_trace_q, s);
  }
  else if (op == 5) autotune_impl<T, ND, VISC, DIAG>(c, qq, oo, 3, s);
  else if (op == 6) jvp_impl<T, ND, VISC, DIAG>(c, qq, vv, nullptr, s, true, (double*)out);
  else jvp_impl<T, ND, VISC, DIAG>(c, qq, vv, oo, s, true);
}

// The instantiations live in one translation unit per (precision, dimension,
// metric) so that they compile in parallel.
#define FR_RUN_CFG(NAME, T, ND, DIAG)                                                             \
  void NAME(fr_ctx* c, int op, const void* q, const void* v, void* out, cudaStream_t s) {        \
    if (c->visc) run_op_cfg<T, ND, true, DIAG>(c, op, q, v, out, s);                           \
    else run_op_cfg<T, ND, false, DIAG>(c, op, q, v, out, s);                                  \
  }

// The double-float residual of one configuration (q: the FP64 state).
#define FR_RUN_RES_DF(NAME, ND, DIAG)                                                              \
  void NAME(fr_ctx* c, const void* q, double* R, cudaStream_t s) {                                  \
    if (c->visc) residual_out64_impl<dfloat, ND, true, DIAG>(c, (const dfloat*)q, R, s);          \
    else residual_out64_impl<dfloat, ND, false, DIAG>(c, (const dfloat*)q, R, s);                 \
  }

}  // namespace frgb
