// Device kernels of the FR residual and its exact JVP (Sec. 2.2).
//
// Data layout (all buckets share it; P = p+1, NSP = P^ND, NFP = P^(ND-1)):
//   state   [element][var][sp]                 sp = i0 + P*i1 + P*P*i2 (xi fastest)
//   trace   [element][face][comp][fp]          comp < NV: q at the face point;
//                                              NV + j*NV + v: physical gradient d_j q_v
//   fout    [element][face][comp][fp]          comp < NV: common transformed flux
//                                              F~_d^com; NV..2NV-1: dq = q^com - q;
//                                              (JVP: 0..NV-1 tangent F~^com, NV.. primal
//                                              dq, 2NV.. tangent dq)
// Face point fp = ia + P*ib, (ia, ib) the tangential directions in increasing
// order.  Element-face blocks have fixed strides (NVT*NFP and 3*NV*NFP values).
#pragma once

#include "fr_internal.h"
#include "physics.cuh"

namespace frgb {

template <int ND, int P>
struct Shape {
  static constexpr int NV = ND + 2;
  static constexpr int NF = 2 * ND;
  static constexpr int NSP = ND == 2 ? P * P : P * P * P;
  static constexpr int NFP = ND == 2 ? P : P * P;
};

// solution point index on face (d, s) line: given face point t and position k along d
template <int ND, int P>
__device__ __forceinline__ int line_sp(int d, int t, int k) {
  if (ND == 2) {
    return d == 0 ? (k + P * t) : (t + P * k);
  } else {
    int a = t % P, b = t / P;
    if (d == 0) return k + P * (a + P * b);
    if (d == 1) return a + P * (k + P * b);
    return a + P * (b + P * k);
  }
}

// face point index (face direction d) of a solution point with indices i[]
template <int ND, int P>
__device__ __forceinline__ int face_pt(int d, const int* i) {
  if (ND == 2) return d == 0 ? i[1] : i[0];
  if (d == 0) return i[1] + P * i[2];
  if (d == 1) return i[0] + P * i[2];
  return i[0] + P * i[1];
}

// runtime versions for the face kernels
__device__ __forceinline__ int orient_map(int code, int t, int P, int nd) {
  int u, v;
  if (nd == 2) {
    u = t;
    v = 0;
  } else {
    int ia = t % P, ib = t / P;
    if (code & 1) {
      u = ib;
      v = ia;
    } else {
      u = ia;
      v = ib;
    }
  }
  if (code & 2) u = P - 1 - u;
  if ((code & 4) && nd == 3) v = P - 1 - v;
  return u + P * v;
}
__device__ __forceinline__ int orient_inv(int code, int uu, int P, int nd) {
  int u = uu % P, v = uu / P;
  if (nd == 2) v = 0;
  if (code & 2) u = P - 1 - u;
  if ((code & 4) && nd == 3) v = P - 1 - v;
  int ia, ib;
  if (nd == 3 && (code & 1)) {
    ia = v;
    ib = u;
  } else {
    ia = u;
    ib = v;
  }
  return ia + P * ib;
}

// State value i: for the double-float kernels the state pointer holds the FP64
// state, converted on load (the FP64 pipe is otherwise idle in those kernels).
template <typename T>
__device__ __forceinline__ T load_state(const T* q, int64_t i) {
  if constexpr (is_dfloat<T>::value) return to_dfloat(reinterpret_cast<const double*>(q)[i]);
  else return q[i];
}

// Gate of a device-driven GMRES cycle (null elsewhere): the launches of the
// cycle's Arnoldi products read it on entry and return at once when it is set,
// which the device-side Givens step does when the cycle has converged.  The
// word is written by an earlier kernel of the same stream and only read here;
// nothing waits on it.
__device__ __forceinline__ bool gate_closed(const int* gate) { return gate != nullptr && *gate != 0; }

template <typename T>
__device__ __forceinline__ T geo_vol(const GeoView<T>& g, int64_t e, int k, int sp) {
  return g.vol[e * g.ves + (int64_t)k * g.vks + (int64_t)sp * g.vps];
}
template <typename T>
__device__ __forceinline__ T geo_face(const GeoView<T>& g, int64_t e, int f, int k, int t) {
  return g.face[e * g.fes + (int64_t)f * g.ffs + (int64_t)k * g.fks + (int64_t)t * g.fps];
}

// ---------------------------------------------------------------------------
// Trace kernel: q (and for NS the physical gradient) at every face point.
// One thread per (element, face, face point).
// ---------------------------------------------------------------------------
template <typename T>
struct TraceArgs {
  const T* q;            // double-float kernels: the FP64 state (see load_state)
  T* trace;
  const int32_t* slot_elem;
  const BasisTab<T>* basis;
  GeoView<T> geo;
  int64_t state_base, trace_base;
  int count, slot_begin, nvt;
  const int* gate = nullptr;   // see gate_closed
};

template <int ND, int P>
struct VolCfg {
  static constexpr int NSP = Shape<ND, P>::NSP;
  static constexpr int EPB = NSP >= 256 ? 1 : 256 / NSP;
  static constexpr int THREADS = EPB * NSP;
};

// One thread per solution point for the load, then per face point: the q
// trace is extrapolated along the normal line (P terms), the normal
// derivative uses l'(+-1) (P terms), and the two tangential derivatives
// differentiate the face trace (P terms each); the physical gradient follows
// from the face metric terms.
// Elements i0 .. i0+epb-1 of the bucket described by ``a``; every thread of the
// block reaches the barriers (threads beyond epb*NSP only help to synchronise).
// DIAG: every metric S is diagonal (axis-aligned affine elements): only S[d][d]
// is read and the metric products reduce to one multiply per component.
// P consecutive values of shared memory (a line with stride 1): 16- or 8-byte
// vector loads when the line's length and every offset that places it (the
// caller's) are multiples of the vector, else scalar loads.
template <typename T, int P, int W>
__device__ __forceinline__ void load_contig(const T* p, T (&x)[P]) {
  constexpr int BYTES = P * (int)sizeof(T);
  if constexpr (W == 16 && BYTES % 16 == 0) {
#pragma unroll
    for (int w = 0; w < BYTES / 16; ++w) {
      const float4 v = reinterpret_cast<const float4*>(p)[w];
      memcpy(reinterpret_cast<char*>(&x[0]) + 16 * w, &v, 16);
    }
  } else if constexpr (W >= 8 && BYTES % 8 == 0) {
#pragma unroll
    for (int w = 0; w < BYTES / 8; ++w) {
      const float2 v = reinterpret_cast<const float2*>(p)[w];
      memcpy(reinterpret_cast<char*>(&x[0]) + 8 * w, &v, 8);
    }
  } else {
#pragma unroll
    for (int k = 0; k < P; ++k) x[k] = p[k];
  }
}

template <typename T, int ND, int P, bool VISC, bool DIAG = false>
__device__ __forceinline__ void trace_body(const TraceArgs<T>& a, int64_t i0, int epb, unsigned char* smem_raw) {
  using Sh = Shape<ND, P>;
  constexpr int NV = Sh::NV, NF = Sh::NF, NSP = Sh::NSP, NFP = Sh::NFP;
  constexpr int NFPT = NF * NFP;                         // face points of an element
  constexpr int ITERS = (NFPT + NSP - 1) / NSP;          // face points per thread, at most
  constexpr int ESTRIDE = NV * NSP + NF * NV * NFP;      // values per element in shared memory
  // widest vector load every contiguous line start is aligned to (element,
  // variable and line offsets; the buffer itself is 16-byte aligned)
  constexpr int SZ = (int)sizeof(T);
  constexpr int W = ((ESTRIDE * SZ) % 16 == 0 && (NSP * SZ) % 16 == 0 && (NFP * SZ) % 16 == 0 && (P * SZ) % 16 == 0)
                        ? 16
                        : (((ESTRIDE * SZ) % 8 == 0 && (NSP * SZ) % 8 == 0 && (NFP * SZ) % 8 == 0 && (P * SZ) % 8 == 0)
                               ? 8
                               : 1);
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int le = threadIdx.x / NSP;
  const int lt = threadIdx.x % NSP;
  const int64_t i = i0 + le;
  const bool valid = le < epb && i < a.count;
  T* sq = sm + le * ESTRIDE;                        // [NV][NSP]
  T* sqf = sq + NV * NSP;                           // [NF][NV][NFP]
  const BasisTab<T>& B = a.basis[P];
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sq[v * NSP + lt] = load_state(a.q, a.state_base + (i * NV + v) * NSP + lt);
  }
  __syncthreads();
  T* out = a.trace + a.trace_base + (valid ? i * NF * (int64_t)a.nvt * NFP : 0);
  // the line values give the trace and (NS) the normal derivative at once;
  // the derivatives wait in registers for the gradient pass
  T dn[ITERS][NV];
  if (valid) {
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
      const int fp = lt + it * NSP;
      if (fp >= NFPT) break;
      const int f = fp / NFP, t = fp % NFP, d = f >> 1, s = f & 1;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T x[P];
        if (d == 0) load_contig<T, P, W>(sq + v * NSP + line_sp<ND, P>(0, t, 0), x);   // stride 1 along xi
        else {
#pragma unroll
          for (int k = 0; k < P; ++k) x[k] = sq[v * NSP + line_sp<ND, P>(d, t, k)];
        }
        Acc<T> ac = acc_init(T(0));
#pragma unroll
        for (int k = 0; k < P; ++k) acc_madd(ac, B.ext[s][k], x[k]);
        const T acc = acc_value(ac);
        out[(f * a.nvt + v) * NFP + t] = acc;
        if (VISC) {
          sqf[(f * NV + v) * NFP + t] = acc;
          Acc<T> an = acc_init(T(0));
#pragma unroll
          for (int k = 0; k < P; ++k) acc_madd(an, B.dext[s][k], x[k]);
          dn[it][v] = acc_value(an);
        }
      }
    }
  }
  if (!VISC) return;
  __syncthreads();
  if (!valid) return;
  const int64_t e = a.slot_elem[a.slot_begin + i];
#pragma unroll
  for (int it = 0; it < ITERS; ++it) {
    const int fp = lt + it * NSP;
    if (fp >= NFPT) break;
    const int f = fp / NFP, t = fp % NFP, d = f >> 1;
    const int ia = t % P, ib = ND == 3 ? t / P : 0;
    const int ta = d == 0 ? 1 : 0;              // first tangential direction (the second is the remaining axis)
    T Sf[ND][ND];
#pragma unroll
    for (int dd = 0; dd < ND; ++dd)
#pragma unroll
      for (int j = 0; j < ND; ++j) Sf[dd][j] = (DIAG && dd != j) ? T(0) : geo_face(a.geo, e, f, dd * ND + j, t);
    const T Jinv = geo_face(a.geo, e, f, ND * ND + 1, t);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* face = sqf + (f * NV + v) * NFP;
      T y[P];
      load_contig<T, P, W>(face + (ND == 2 ? 0 : P * ib), y);   // the face line along its first axis
      Acc<T> ac = acc_init(T(0));
#pragma unroll
      for (int m = 0; m < P; ++m) acc_madd(ac, B.D[ia][m], y[m]);
      const T da = acc_value(ac);
      T db = T(0);
      if (ND == 3) {
        ac = acc_init(T(0));
#pragma unroll
        for (int m = 0; m < P; ++m) acc_madd(ac, B.D[ib][m], face[ia + P * m]);
        db = acc_value(ac);
      }
      // reference derivatives by axis through selects on the face's axes (a
      // register array indexed by d / ta / tb would be placed in local memory)
      T dq[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) dq[j] = j == d ? dn[it][v] : (j == ta ? da : db);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        T g = T(0);
        if (DIAG) {
          g = Sf[j][j] * dq[j];
        } else {
#pragma unroll
          for (int dd = 0; dd < ND; ++dd) g = madd(g, Sf[dd][j], dq[dd]);
        }
        out[(f * a.nvt + NV + j * NV + v) * NFP + t] = g * Jinv;
      }
    }
  }
}

template <typename T, int ND, int P, bool VISC, bool DIAG>
__global__ void __launch_bounds__(256) trace_kernel(TraceArgs<T> a, int epb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(a.gate)) return;
  trace_body<T, ND, P, VISC, DIAG>(a, (int64_t)blockIdx.x * epb, epb, smem_raw);
}

constexpr int kMaxBuckets = kMaxDeg + 1;

template <typename T>
struct TraceMulti {
  TraceArgs<T> b[kMaxBuckets];
  int P[kMaxBuckets];
  int epb[kMaxBuckets];
  const WorkItem* items;
  int n_items;
};

// Every bucket in one persistent launch: CTAs walk the cost-ordered work
// table with a grid stride and dispatch on the tile's degree.
template <typename T, int ND, bool VISC, bool DIAG>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) trace_multi_kernel(const __grid_constant__ TraceMulti<T> m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(m.b[0].gate)) return;
  for (int w = blockIdx.x; w < m.n_items; w += gridDim.x) {
    const WorkItem it = m.items[w];
    const int b = it.bucket;
    switch (m.P[b]) {
      case 2: trace_body<T, ND, 2, VISC, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
      case 3: trace_body<T, ND, 3, VISC, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
      case 4: trace_body<T, ND, 4, VISC, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
      case 5: trace_body<T, ND, 5, VISC, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
      case 6: trace_body<T, ND, 6, VISC, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Interior face kernel: common flux on the mortar (Pm points per direction).
// One thread per (face, mortar point).  MODE 0: residual; 1: JVP.
// ---------------------------------------------------------------------------
template <typename T>
struct FaceArgs {
  const FaceRec* recs;
  const T* trq;        // traces of q
  const T* trv;        // traces of the tangent (JVP)
  T* fout;
  T* scratch;          // mixed-degree groups: [face][comp][NFPm]
  const BasisTab<T>* basis;
  const MortarTab<T>* mortar;   // Pm -> Ps tables (nullptr when Pm == Ps)
  GeoView<T> geo_m, geo_s;
  T gamma, mu, kappa;
  int n, Pm, Ps, nvt;
  int flux;            // common inviscid flux: 0 Rusanov, 1 Roe
  int64_t scratch_base;
  const int* gate = nullptr;   // see gate_closed
};

template <int ND, typename S, typename T>
__device__ __forceinline__ void load_trace_pt(const T* trq, const T* trv, int64_t base, int comp0,
                                              int ncomp, int NFP, int t, S* out) {
  for (int c = 0; c < ncomp; ++c) {
    T v = trq[base + (int64_t)(comp0 + c) * NFP + t];
    T dv = trv ? trv[base + (int64_t)(comp0 + c) * NFP + t] : T(0);
    set_scalar(out[c], v, dv);
  }
}

// value of the slave's trace component at mortar point u (slave axes, Pm grid)
template <int ND, typename S, typename T>
__device__ __forceinline__ void slave_at_mortar(const FaceArgs<T>& a, int64_t base, int comp0,
                                                int ncomp, int u, S* out) {
  const int Ps = a.Ps, Pm = a.Pm;
  const int NFPs = ND == 2 ? Ps : Ps * Ps;
  if (Pm == Ps) {
    load_trace_pt<ND>(a.trq, a.trv, base, comp0, ncomp, NFPs, u, out);
    return;
  }
  const int ua = u % Pm, ub = ND == 2 ? 0 : u / Pm;
  for (int c = 0; c < ncomp; ++c) set_scalar(out[c], T(0), T(0));
  for (int bb = 0; bb < (ND == 2 ? 1 : Ps); ++bb) {
    const T wb = ND == 2 ? T(1) : a.mortar->I[ub][bb];
    for (int aa = 0; aa < Ps; ++aa) {
      const T w = a.mortar->I[ua][aa] * wb;
      const int pt = aa + Ps * bb;
      for (int c = 0; c < ncomp; ++c) {
        T v = a.trq[base + (int64_t)(comp0 + c) * NFPs + pt];
        T dv = a.trv ? a.trv[base + (int64_t)(comp0 + c) * NFPs + pt] : T(0);
        S x;
        set_scalar(x, v, dv);
        out[c] = out[c] + w * x;
      }
    }
  }
}

template <int ND, typename T>
__device__ __forceinline__ void slave_coef_at_mortar(const FaceArgs<T>& a, const FaceRec& r, int u,
                                                     T* cS) {
  // c = g_s'(face) S_d[j] / |J| at the slave's own points, interpolated to the mortar
  const int Ps = a.Ps, Pm = a.Pm;
  const int ds = r.sf >> 1, ss = r.sf & 1;
  const T g = a.basis[Ps].dgf[ss];
  for (int j = 0; j < ND; ++j) cS[j] = T(0);
  if (Pm == Ps) {
    const T gJ = g * geo_face(a.geo_s, r.se, r.sf, ND * ND + 1, u);
    for (int j = 0; j < ND; ++j) cS[j] = gJ * geo_face(a.geo_s, r.se, r.sf, ds * ND + j, u);
    return;
  }
  const int ua = u % Pm, ub = ND == 2 ? 0 : u / Pm;
  for (int bb = 0; bb < (ND == 2 ? 1 : Ps); ++bb) {
    const T wb = ND == 2 ? T(1) : a.mortar->I[ub][bb];
    for (int aa = 0; aa < Ps; ++aa) {
      const T w = a.mortar->I[ua][aa] * wb;
      const int pt = aa + Ps * bb;
      const T gJ = g * geo_face(a.geo_s, r.se, r.sf, ND * ND + 1, pt);
      for (int j = 0; j < ND; ++j) cS[j] += w * (gJ * geo_face(a.geo_s, r.se, r.sf, ds * ND + j, pt));
    }
  }
}

// DIAG: both sides have diagonal metrics (axis-aligned affine elements), so the
// area vector and the BR2 lifting coefficients point along the master face's
// axis dm and only the viscous flux row dm is needed.  Face records are sorted
// by dm, so the branches on it are warp-uniform.
// FP32 and double-float: four CTAs an SM (128 registers).  Uncapped, the
// FP32 JVP instance for general metrics held 183 registers (two CTAs); the
// double-float viscous instance spills 160 bytes at the cap and still streams
// its traces faster than at three CTAs (252 -> 234 us at 32^3).
template <typename T, int ND, bool VISC, int MODE, bool DIAG = false>
__global__ void __launch_bounds__(128, (is_dfloat<T>::value || sizeof(T) == 4) ? 4 : 1) face_kernel(FaceArgs<T> a) {
  constexpr int NV = ND + 2;
  if (gate_closed(a.gate)) return;
  using S = typename std::conditional<MODE == 1, Dual<T>, T>::type;
  const int Pm = a.Pm;
  const int NFPm = ND == 2 ? Pm : Pm * Pm;
  const int NFPs = ND == 2 ? a.Ps : a.Ps * a.Ps;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)a.n * NFPm) return;
  const int t = (int)(gid % NFPm);
  const FaceRec r = a.recs[gid / NFPm];
  const int dm = r.mf >> 1, sm = r.mf & 1, ss = r.sf & 1;
  const int u = orient_map(r.orient, t, Pm, ND);
  const T* trv = MODE == 1 ? a.trv : nullptr;

  S qM[NV], qS[NV];
  load_trace_pt<ND>(a.trq, trv, r.mt, 0, NV, NFPm, t, qM);
  {
    FaceArgs<T> b = a;
    b.trv = trv;
    slave_at_mortar<ND>(b, r.st, 0, NV, u, qS);
  }
  T A[ND], n[ND];
  const T sgm = sm ? T(1) : T(-1);
  const T absA = geo_face(a.geo_m, r.me, r.mf, ND * ND + 2 + dm, t);
  const T inv_absA = geo_face(a.geo_m, r.me, r.mf, ND * ND + 2 + ND + dm, t);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    A[j] = sgm * geo_face(a.geo_m, r.me, r.mf, dm * ND + j, t);
    n[j] = A[j] * inv_absA;
  }
  S Fn[NV];
  common_flux<ND>(a.flux, qM, qS, n, absA, a.gamma, Fn);
  S qc[NV];
  if (VISC) {
#pragma unroll
    for (int v = 0; v < NV; ++v) qc[v] = T(0.5) * (qM[v] + qS[v]);
    T cM[ND], cS[ND];
    const T gJ = a.basis[Pm].dgf[sm] * geo_face(a.geo_m, r.me, r.mf, ND * ND + 1, t);
#pragma unroll
    for (int j = 0; j < ND; ++j) cM[j] = gJ * geo_face(a.geo_m, r.me, r.mf, dm * ND + j, t);
    slave_coef_at_mortar<ND>(a, r, u, cS);
    S GM[ND][NV], GS[ND][NV], Gc[ND][NV];
    load_trace_pt<ND>(a.trq, trv, r.mt, NV, ND * NV, NFPm, t, &GM[0][0]);
    {
      FaceArgs<T> b = a;
      b.trv = trv;
      slave_at_mortar<ND>(b, r.st, NV, ND * NV, u, &GS[0][0]);
    }
    if (DIAG) {
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) Gc[j][v] = T(0.5) * (GM[j][v] + GS[j][v]);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        if (j != dm) continue;
#pragma unroll
        for (int v = 0; v < NV; ++v) Gc[j][v] = Gc[j][v] + T(0.5) * (cM[j] * (qc[v] - qM[v]) + cS[j] * (qc[v] - qS[v]));
      }
      S fr[NV];
      flux_viscous_row<ND>(qc, Gc, a.gamma, a.mu, a.kappa, dm, fr);
      T Ad = T(0);
#pragma unroll
      for (int j = 0; j < ND; ++j)
        if (j == dm) Ad = A[j];
#pragma unroll
      for (int v = 0; v < NV; ++v) Fn[v] = Fn[v] - fr[v] * Ad;
    } else {
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v)
          Gc[j][v] = T(0.5) * (GM[j][v] + cM[j] * (qc[v] - qM[v]) + GS[j][v] + cS[j] * (qc[v] - qS[v]));
      S fv[ND][NV];
      flux_viscous<ND>(qc, Gc, a.gamma, a.mu, a.kappa, fv);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        S acc = szero<S>();
#pragma unroll
        for (int j = 0; j < ND; ++j) acc = acc + fv[j][v] * A[j];
        Fn[v] = Fn[v] - acc;
      }
    }
  }
  // master side
  T* om = a.fout + r.mo;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    S x = sgm * Fn[v];
    om[v * NFPm + t] = MODE == 1 ? tangent(x) : value(x);
    if (VISC) {
      S dq = qc[v] - qM[v];
      om[(NV + v) * NFPm + t] = value(dq);
      if (MODE == 1) om[(2 * NV + v) * NFPm + t] = tangent(dq);
    }
  }
  const T sgs = ss ? T(1) : T(-1);
  if (Pm == a.Ps) {
    T* os = a.fout + r.so;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      S x = sgs * (T(0) - Fn[v]);
      os[v * NFPs + u] = MODE == 1 ? tangent(x) : value(x);
      if (VISC) {
        S dq = qc[v] - qS[v];
        os[(NV + v) * NFPs + u] = value(dq);
        if (MODE == 1) os[(2 * NV + v) * NFPs + u] = tangent(dq);
      }
    }
  } else {
    // mortar values (master order) for the projection kernel: -Fn, then q^com
    T* sc = a.scratch + a.scratch_base + (int64_t)r.idx * 4 * NV * NFPm;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      S x = T(0) - Fn[v];
      sc[v * NFPm + t] = MODE == 1 ? tangent(x) : value(x);
      if (VISC) {
        sc[(NV + v) * NFPm + t] = value(qc[v]);
        if (MODE == 1) sc[(2 * NV + v) * NFPm + t] = tangent(qc[v]);
      }
    }
  }
}

// L2 projection of the mortar values onto the lower-degree side.
// One thread per (face, slave point).
template <typename T, int ND, bool VISC, int MODE>
__global__ void __launch_bounds__(128) mortar_project_kernel(FaceArgs<T> a) {
  constexpr int NV = ND + 2;
  if (gate_closed(a.gate)) return;
  const int Pm = a.Pm, Ps = a.Ps;
  const int NFPm = ND == 2 ? Pm : Pm * Pm;
  const int NFPs = ND == 2 ? Ps : Ps * Ps;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)a.n * NFPs) return;
  const int pt = (int)(gid % NFPs);
  const FaceRec r = a.recs[gid / NFPs];
  const int ss = r.sf & 1;
  const T sgs = ss ? T(1) : T(-1);
  const int pa = pt % Ps, pb = ND == 2 ? 0 : pt / Ps;
  const T* sc = a.scratch + a.scratch_base + (int64_t)r.idx * 4 * NV * NFPm;
  const int ncomp = VISC ? (MODE == 1 ? 3 * NV : 2 * NV) : NV;
  T acc[3 * NV];
  for (int c = 0; c < ncomp; ++c) acc[c] = T(0);
  for (int mb = 0; mb < (ND == 2 ? 1 : Pm); ++mb) {
    const T wb = ND == 2 ? T(1) : a.mortar->Pi[pb][mb];
    for (int ma = 0; ma < Pm; ++ma) {
      const T w = a.mortar->Pi[pa][ma] * wb;
      const int tm = orient_inv(r.orient, ma + Pm * mb, Pm, ND);
      for (int c = 0; c < ncomp; ++c) acc[c] += w * sc[c * NFPm + tm];
    }
  }
  T* os = a.fout + r.so;
  for (int v = 0; v < NV; ++v) {
    os[v * NFPs + pt] = sgs * acc[v];
    if (VISC) {
      const T qs = a.trq[r.st + (int64_t)v * NFPs + pt];
      os[(NV + v) * NFPs + pt] = acc[NV + v] - qs;
      if (MODE == 1) {
        const T qsd = a.trv[r.st + (int64_t)v * NFPs + pt];
        os[(2 * NV + v) * NFPs + pt] = acc[2 * NV + v] - qsd;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Boundary faces: ghost state (wall / far field).  One thread per (face, point).
// ---------------------------------------------------------------------------
template <typename T>
struct BndArgs {
  const BndRec* recs;
  const T* trq;
  const T* trv;
  T* fout;
  const BasisTab<T>* basis;
  GeoView<T> geo;
  T gamma, mu, kappa;
  T qinf[5];
  int n, P, kind;
  int flux;            // common inviscid flux: 0 Rusanov, 1 Roe
  const int* gate = nullptr;   // see gate_closed
};

template <typename T, int ND, bool VISC, int MODE>
__global__ void __launch_bounds__(128) bnd_kernel(BndArgs<T> a) {
  constexpr int NV = ND + 2;
  if (gate_closed(a.gate)) return;
  using S = typename std::conditional<MODE == 1, Dual<T>, T>::type;
  const int P = a.P;
  const int NFP = ND == 2 ? P : P * P;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)a.n * NFP) return;
  const int t = (int)(gid % NFP);
  const BndRec r = a.recs[gid / NFP];
  const int d = r.mf >> 1, s = r.mf & 1;
  const T* trv = MODE == 1 ? a.trv : nullptr;
  S qM[NV], qG[NV];
  load_trace_pt<ND>(a.trq, trv, r.mt, 0, NV, NFP, t, qM);
  ghost_state<ND>(qM, a.kind, a.qinf, qG);
  T A[ND], n[ND];
  const T sg = s ? T(1) : T(-1);
  const T absA = geo_face(a.geo, r.me, r.mf, ND * ND + 2 + d, t);
  const T inv_absA = geo_face(a.geo, r.me, r.mf, ND * ND + 2 + ND + d, t);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    A[j] = sg * geo_face(a.geo, r.me, r.mf, d * ND + j, t);
    n[j] = A[j] * inv_absA;
  }
  S Fn[NV];
  common_flux<ND>(a.flux, qM, qG, n, absA, a.gamma, Fn);
  S qc[NV];
  if (VISC) {
#pragma unroll
    for (int v = 0; v < NV; ++v) qc[v] = T(0.5) * (qM[v] + qG[v]);
    T cM[ND];
    const T gJ = a.basis[P].dgf[s] * geo_face(a.geo, r.me, r.mf, ND * ND + 1, t);
#pragma unroll
    for (int j = 0; j < ND; ++j) cM[j] = gJ * geo_face(a.geo, r.me, r.mf, d * ND + j, t);
    S GM[ND][NV], Gc[ND][NV];
    load_trace_pt<ND>(a.trq, trv, r.mt, NV, ND * NV, NFP, t, &GM[0][0]);
#pragma unroll
    for (int j = 0; j < ND; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) Gc[j][v] = GM[j][v] + cM[j] * (qc[v] - qM[v]);
    S fv[ND][NV];
    flux_viscous<ND>(qc, Gc, a.gamma, a.mu, a.kappa, fv);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      S acc = szero<S>();
#pragma unroll
      for (int j = 0; j < ND; ++j) acc = acc + fv[j][v] * A[j];
      if (a.kind == -1 && v == NV - 1) acc = szero<S>();   // adiabatic wall
      Fn[v] = Fn[v] - acc;
    }
  }
  T* om = a.fout + r.mo;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    S x = sg * Fn[v];
    om[v * NFP + t] = MODE == 1 ? tangent(x) : value(x);
    if (VISC) {
      S dq = qc[v] - qM[v];
      om[(NV + v) * NFP + t] = value(dq);
      if (MODE == 1) om[(2 * NV + v) * NFP + t] = tangent(dq);
    }
  }
}

// ---------------------------------------------------------------------------
// Volume kernel: corrected gradient, flux, divergence and FR correction.
// One thread per solution point, EPB elements per block.
// ---------------------------------------------------------------------------
template <typename T>
struct VolArgs {
  const T* q;          // double-float kernels: the FP64 state (see load_state)
  const T* v;          // tangent (JVP)
  T* out;
  double* out_neg64;   // JVP only, optional: -J v written in FP64 instead of out
  double* out64;       // double-float residual: R written in FP64 (out unused)
  const T* fout;
  const int32_t* slot_elem;
  const BasisTab<T>* basis;
  GeoView<T> geo;
  T gamma, mu, kappa;
  int64_t state_base, out_base;
  int count, slot_begin;
  const int* gate = nullptr;   // see gate_closed
  // JVP, optional: J v is multiplied by *vscale (v is a stored Krylov column
  // whose scale lives on the device; J is linear in v)
  const double* vscale = nullptr;
};


template <typename T, int ND, int P, bool VISC, int MODE, bool DIAG = false>
__device__ __forceinline__ void vol_body(const VolArgs<T>& a, int64_t i0, int epb, unsigned char* smem_raw) {
  using Sh = Shape<ND, P>;
  using S = typename std::conditional<MODE == 1, Dual<T>, T>::type;
  constexpr int NV = Sh::NV, NF = Sh::NF, NSP = Sh::NSP, NFP = Sh::NFP;
  constexpr int FOUT_STRIDE = 3 * NV * NFP;
  S* sm = reinterpret_cast<S*>(smem_raw);
  const int le = threadIdx.x / NSP;
  const int sp = threadIdx.x % NSP;
  const int64_t i = i0 + le;
  const bool valid = le < epb && i < a.count;
  S* sq = sm + le * (NV + ND * NV) * NSP;       // [NV][NSP]
  S* sF = sq + NV * NSP;                         // [ND][NV][NSP]
  const BasisTab<T>& B = a.basis[P];
  int idx[3];
  idx[0] = sp % P;
  idx[1] = (sp / P) % P;
  idx[2] = ND == 3 ? sp / (P * P) : 0;
  const int64_t e = valid ? a.slot_elem[a.slot_begin + i] : 0;
  const T* fo = a.fout + (valid ? a.out_base + i * NF * FOUT_STRIDE : 0);
  // JVP: the element's face outputs (contiguous, NF blocks) prefetched into
  // L1 line by line before the state loads; every solution point reads its
  // lines' values with scalar loads later, which then hit L1 (the FP32 JVP
  // volume kernel waited on these loads: 119 -> 110 us at 32^3)
  if (MODE == 1 && valid) {
    constexpr int LINE = 128 / (int)sizeof(T);   // values of a 128-byte line
    for (int o = sp * LINE; o < NF * FOUT_STRIDE; o += NSP * LINE)
      asm volatile("prefetch.global.L1 [%0];" ::"l"(fo + o));
  }

  S q[NV];
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T x = load_state(a.q, a.state_base + (i * NV + v) * NSP + sp);
      T dx = MODE == 1 ? a.v[a.state_base + (i * NV + v) * NSP + sp] : T(0);
      set_scalar(q[v], x, dx);
      sq[v * NSP + sp] = q[v];
    }
  }
  __syncthreads();

  T Sm[ND][ND];
  T Jinv = T(1);
  if (valid) {
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int j = 0; j < ND; ++j) Sm[d][j] = (DIAG && d != j) ? T(0) : geo_vol(a.geo, e, d * ND + j, sp);
    Jinv = geo_vol(a.geo, e, ND * ND + 1, sp);

    S f[ND][NV];
    flux_inviscid<ND>(q, a.gamma, f);
    if (VISC) {
      S gref[ND][NV];
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
        const int base = sp - idx[d] * stride;
        const int tf = face_pt<ND, P>(d, idx);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          Acc<S> acc = acc_init(szero<S>());
#pragma unroll
          for (int k = 0; k < P; ++k) acc_madd(acc, B.D[idx[d]][k], sq[v * NSP + base + k * stride]);
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const T* blk = fo + (2 * d + s) * FOUT_STRIDE;
            S dq;
            set_scalar(dq, blk[(NV + v) * NFP + tf], MODE == 1 ? blk[(2 * NV + v) * NFP + tf] : T(0));
            acc_madd(acc, B.dg[s][idx[d]], dq);
          }
          gref[d][v] = acc_value(acc);
        }
      }
      S G[ND][NV];
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (DIAG) {
            G[j][v] = (Sm[j][j] * Jinv) * gref[j][v];
          } else {
            S acc = szero<S>();
#pragma unroll
            for (int d = 0; d < ND; ++d) acc = acc + Sm[d][j] * gref[d][v];
            G[j][v] = acc * Jinv;
          }
        }
      S fv[ND][NV];
      flux_viscous<ND>(q, G, a.gamma, a.mu, a.kappa, fv);
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) f[j][v] = f[j][v] - fv[j][v];
    }
    // transformed flux F~_d = sum_j S[d][j] f_j
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (DIAG) {
          sF[(d * NV + v) * NSP + sp] = Sm[d][d] * f[d][v];
        } else {
          S acc = szero<S>();
#pragma unroll
          for (int j = 0; j < ND; ++j) acc = acc + Sm[d][j] * f[j][v];
          sF[(d * NV + v) * NSP + sp] = acc;
        }
      }
  }
  __syncthreads();
  if (!valid) return;

  // divergence D_d F~_d plus the correction g_s'(xi_d) (F~^com - F~(xi_d = +-1))
  S div[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) div[v] = szero<S>();
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
    const int base = sp - idx[d] * stride;
    const int tf = face_pt<ND, P>(d, idx);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const S* line = sF + (d * NV + v) * NSP + base;
      Acc<S> acc = acc_init(szero<S>());
#pragma unroll
      for (int k = 0; k < P; ++k) acc_madd(acc, B.Dh[idx[d]][k], line[k * stride]);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        S com;
        const T c = fo[(2 * d + s) * FOUT_STRIDE + v * NFP + tf];
        if (MODE == 1) set_scalar(com, T(0), c); else set_scalar(com, c, T(0));
        acc_madd(acc, B.dg[s][idx[d]], com);
      }
      div[v] = div[v] + acc_value(acc);
    }
  }
  const double vs = (MODE == 1 && a.vscale) ? *a.vscale : 1.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    S r = (T(0) - div[v]) * Jinv;
    if constexpr (is_dfloat<T>::value) {
      a.out64[a.state_base + (i * NV + v) * NSP + sp] = to_double(value(r));
    } else {
      if (MODE == 1 && a.out_neg64)
        a.out_neg64[a.state_base + (i * NV + v) * NSP + sp] = -vs * (double)tangent(r);
      else if (MODE == 1)
        a.out[a.state_base + (i * NV + v) * NSP + sp] = a.vscale ? (T)vs * tangent(r) : tangent(r);
      else
        a.out[a.state_base + (i * NV + v) * NSP + sp] = value(r);
    }
  }
}

template <typename T, int ND, int P, bool VISC, int MODE, bool DIAG>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : (is_dfloat<T>::value ? 2 : 1)) vol_kernel(VolArgs<T> a, int epb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(a.gate)) return;
  vol_body<T, ND, P, VISC, MODE, DIAG>(a, (int64_t)blockIdx.x * epb, epb, smem_raw);
}

template <typename T>
struct VolMulti {
  VolArgs<T> b[kMaxBuckets];
  int P[kMaxBuckets];
  int epb[kMaxBuckets];
  const WorkItem* items;
  int n_items;
};

template <typename T, int ND, bool VISC, int MODE, bool DIAG>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 || is_dfloat<T>::value) ? 2 : 1) vol_multi_kernel(const __grid_constant__ VolMulti<T> m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(m.b[0].gate)) return;
  for (int w = blockIdx.x; w < m.n_items; w += gridDim.x) {
    const WorkItem it = m.items[w];
    const int b = it.bucket;
    switch (m.P[b]) {
      case 2: vol_body<T, ND, 2, VISC, MODE, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
      case 3: vol_body<T, ND, 3, VISC, MODE, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
      case 4: vol_body<T, ND, 4, VISC, MODE, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
      case 5: vol_body<T, ND, 5, VISC, MODE, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
      case 6: vol_body<T, ND, 6, VISC, MODE, DIAG>(m.b[b], it.first, m.epb[b], smem_raw); break;
    }
    __syncthreads();
  }
}

}  // namespace frgb
