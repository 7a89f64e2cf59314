// Fused exact JVP (Sec. 2.2 differentiated; the GMRES product of Sec. 2.3) for
// meshes whose faces are all interior and conforming (the same degree on both
// sides, no boundary): the Taylor-Green and Fourier-mode boxes, periodic
// vortices and batches of them.
//
// Two passes instead of three:
//   1. compact traces: q and its reference normal derivative at every face
//      point (2 NV values, against NV (1 + ND) for the trace-gradient layout),
//      written once per Newton iteration for q and once per product for v;
//   2. one kernel per element tile: the element's own traces are rebuilt on
//      chip from its solution points, the neighbours' compact traces of the
//      shared faces are gathered from global memory, the tangential
//      derivatives of both sides are formed from the face traces, and the
//      common flux, BR2 gradient and lifting are evaluated at every face point
//      of the element in the master's orientation (master and slave as the
//      face records define them), so that both sides of a face evaluate the
//      same expression on the same values and receive exactly opposite fluxes;
//      the corrected gradient, fluxes, divergence and correction follow from
//      the face outputs kept in shared memory.
// No face-output array goes through HBM; the face flux is evaluated twice
// (once from each side), which costs arithmetic instead of bytes.
//
// Layouts: compact traces [slot][face][CT][NFP] (CT = 2 NV for Navier-Stokes:
// q then the normal derivative; NV for Euler), at a per-bucket base.
#pragma once

#include "fr_kernels.cuh"

namespace frgb {

// Explicit fused multiply-adds: the compact traces of q are formed by two
// kernels (the trace pass and, for the element itself, the fused kernel), and
// both sides of a face must see the same bits.
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <bool VISC, int NV>
struct CompactWidth {
  static constexpr int value = VISC ? 2 * NV : NV;
};

// Widest vector load (16, 8 or 1 bytes) that every line along xi of elements
// staged [NV][NSP] at multiples of BLOCK values from a 16-byte aligned base is
// aligned to: the block, variable and line (a multiple of P) offsets.
template <typename T, int P, int NSP, int BLOCK>
constexpr int line_vec_width() {
  constexpr int SZ = (int)sizeof(T);
  return (BLOCK * SZ) % 16 == 0 && (NSP * SZ) % 16 == 0 && (P * SZ) % 16 == 0   ? 16
         : (BLOCK * SZ) % 8 == 0 && (NSP * SZ) % 8 == 0 && (P * SZ) % 8 == 0 ? 8
                                                                              : 1;
}

// q and (Navier-Stokes) the reference normal derivative at face point fp of an
// element staged in shared memory as [NV][NSP]; W > 1: the caller's element is
// W-byte aligned as line_vec_width states, and lines along xi (contiguous) are
// read as vectors (the same values).
template <typename T, int ND, int P, bool VISC, int W = 1>
__device__ __forceinline__ void trace_point(const T* sq, const BasisTab<T>& B, int fp, T* qf, T* dn) {
  using Sh = Shape<ND, P>;
  constexpr int NV = Sh::NV, NSP = Sh::NSP, NFP = Sh::NFP;
  const int f = fp / NFP, t = fp % NFP, d = f >> 1, s = f & 1;
  // the normal line through face point t: solution points base + k stride
  // (its offsets computed once for all variables)
  const int base = line_sp<ND, P>(d, t, 0);
  const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
  int off[P];
#pragma unroll
  for (int k = 0; k < P; ++k) off[k] = base + k * stride;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T x[P];
    if (W > 1 && d == 0) {
      load_contig<T, P, W>(sq + v * NSP + base, x);
    } else {
#pragma unroll
      for (int k = 0; k < P; ++k) x[k] = sq[v * NSP + off[k]];
    }
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < P; ++k) acc = xfma(B.ext[s][k], x[k], acc);
    qf[v] = acc;
    if (VISC) {
      T an = T(0);
#pragma unroll
      for (int k = 0; k < P; ++k) an = xfma(B.dext[s][k], x[k], an);
      dn[v] = an;
    }
  }
}

// ---------------------------------------------------------------------------
// Pass 1: compact traces.  One thread per solution point for the load, then
// per face point.
// ---------------------------------------------------------------------------
template <typename T>
struct CTraceArgs {
  const T* q;
  T* out;
  const BasisTab<T>* basis;
  int64_t state_base, ctrace_base;
  int count;
  const int* gate = nullptr;   // see gate_closed
};

template <typename T, int ND, int P, bool VISC>
__global__ void __launch_bounds__(256) ctrace_kernel(CTraceArgs<T> a, int epb) {
  using Sh = Shape<ND, P>;
  constexpr int NV = Sh::NV, NF = Sh::NF, NSP = Sh::NSP, NFP = Sh::NFP;
  constexpr int CT = CompactWidth<VISC, NV>::value;
  constexpr int NFPT = NF * NFP, ITERS = (NFPT + NSP - 1) / NSP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(a.gate)) return;
  const int le = threadIdx.x / NSP, lt = threadIdx.x % NSP;
  const int64_t i = (int64_t)blockIdx.x * epb + le;
  const bool valid = le < epb && i < a.count;
  T* sq = reinterpret_cast<T*>(smem_raw) + le * NV * NSP;
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sq[v * NSP + lt] = a.q[a.state_base + (i * NV + v) * NSP + lt];
  }
  __syncthreads();
  if (!valid) return;
  const BasisTab<T>& B = a.basis[P];
  T* out = a.out + a.ctrace_base + i * NF * CT * NFP;
#pragma unroll
  for (int it = 0; it < ITERS; ++it) {
    const int fp = lt + it * NSP;
    if (fp >= NFPT) break;
    const int f = fp / NFP, t = fp % NFP;
    T qf[NV], dn[NV];
    trace_point<T, ND, P, VISC, line_vec_width<T, P, NSP, NV * NSP>()>(sq, B, fp, qf, dn);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      out[(f * CT + v) * NFP + t] = qf[v];
      if (VISC) out[(f * CT + NV + v) * NFP + t] = dn[v];
    }
  }
}

// Physical gradient (value and tangent) at point t of face fc from that
// face's compact traces Xq (of q) and Xv (of v), laid out [CT][NFP]: the
// normal derivative is stored, the two tangential derivatives differentiate
// the face trace along its own axes (P terms each), and the face metric terms
// map reference to physical derivatives.
template <typename T, int ND, int P, bool DIAG>
__device__ __forceinline__ void face_metric(const GeoView<T>& geo, int64_t e, int fc, int t, T (&Sf)[ND][ND], T& Jinv) {
#pragma unroll
  for (int dd = 0; dd < ND; ++dd)
#pragma unroll
    for (int j = 0; j < ND; ++j) Sf[dd][j] = (DIAG && dd != j) ? T(0) : geo_face(geo, e, fc, dd * ND + j, t);
  Jinv = geo_face(geo, e, fc, ND * ND + 1, t);
}

template <typename T, int ND, int P, bool DIAG>
__device__ __forceinline__ void face_grad_m(const T* Xq, const T* Xv, int fc, int t, const T (&Sf)[ND][ND], T Jinv,
                                            const BasisTab<T>& B, Dual<T> (*G)[ND + 2]) {
  constexpr int NV = ND + 2;
  constexpr int NFP = ND == 2 ? P : P * P;
  const int dc = fc >> 1;
  const int ia = t % P, ib = ND == 3 ? t / P : 0;
  const int ta = dc == 0 ? 1 : 0;   // first tangential direction (the second is the remaining axis)
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const Dual<T> dn{Xq[(NV + v) * NFP + t], Xv[(NV + v) * NFP + t]};
    const T* yq = Xq + v * NFP;
    const T* yv = Xv + v * NFP;
    T aq = T(0), av = T(0);
#pragma unroll
    for (int m = 0; m < P; ++m) {
      aq = xfma(B.D[ia][m], yq[m + P * ib], aq);
      av = xfma(B.D[ia][m], yv[m + P * ib], av);
    }
    const Dual<T> da{aq, av};
    Dual<T> db{T(0), T(0)};
    if (ND == 3) {
      aq = T(0);
      av = T(0);
#pragma unroll
      for (int m = 0; m < P; ++m) {
        aq = xfma(B.D[ib][m], yq[ia + P * m], aq);
        av = xfma(B.D[ib][m], yv[ia + P * m], av);
      }
      db = Dual<T>{aq, av};
    }
    // reference derivatives by axis, chosen by selects on the face's axes
    // (indexing a register array by dc / ta / tb would place it in local memory)
    Dual<T> dq[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) dq[j] = j == dc ? dn : (j == ta ? da : db);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      Dual<T> g{T(0), T(0)};
      if (DIAG) {
        g = Sf[j][j] * dq[j];
      } else {
#pragma unroll
        for (int dd = 0; dd < ND; ++dd) g = g + Sf[dd][j] * dq[dd];
      }
      G[j][v] = g * Jinv;
    }
  }
}

// The same with the metric terms read here.
template <typename T, int ND, int P, bool DIAG>
__device__ __forceinline__ void face_grad(const T* Xq, const T* Xv, int fc, int t, const GeoView<T>& geo, int64_t e,
                                          const BasisTab<T>& B, Dual<T> (*G)[ND + 2]) {
  T Sf[ND][ND], Jinv;
  face_metric<T, ND, P, DIAG>(geo, e, fc, t, Sf, Jinv);
  face_grad_m<T, ND, P, DIAG>(Xq, Xv, fc, t, Sf, Jinv, B, G);
}

// ---------------------------------------------------------------------------
// Pass 2: faces and volume of a tile of elements.
// ---------------------------------------------------------------------------
template <typename T>
struct FusedArgs {
  const T* q;           // state (bucket layout)
  const T* v;           // tangent
  const T* trq;         // compact traces of q and of v (all buckets)
  const T* trv;
  T* out;               // J v in T, or
  double* out_neg64;    // -J v in FP64 (the Arnoldi vector) when non-null
  const FusedNbr* nbr;  // [slot][NF]
  const int32_t* slot_elem;
  const BasisTab<T>* basis;
  GeoView<T> geo;
  T gamma, mu, kappa;
  int flux;
  int64_t state_base, ctrace_base;
  int count, slot_begin;
  const int* gate = nullptr;   // see gate_closed
  const double* vscale = nullptr;   // optional: J v multiplied by *vscale (see VolArgs)
};

// Shared memory of one element, in values of T: the state and tangent, the
// four compact-trace blocks (own q and v, the neighbours' q and v), which the
// volume fluxes (ND x NV duals a point) reuse once the faces are done, and
// the face outputs.
template <int ND, int P, bool VISC>
struct FusedSmem {
  static constexpr int NV = ND + 2, NF = 2 * ND;
  static constexpr int NSP = Shape<ND, P>::NSP, NFP = Shape<ND, P>::NFP;
  static constexpr int CT = CompactWidth<VISC, NV>::value;
  static constexpr int TB = NF * CT * NFP;                     // compact traces of one element (q or v)
  static constexpr int FO = (VISC ? 3 : 1) * NV * NFP;         // face outputs of one face
  static constexpr int REG = 4 * TB > 2 * ND * NV * NSP ? 4 * TB : 2 * ND * NV * NSP;
  static constexpr int PER = 2 * NV * NSP + REG + NF * FO;
};

template <typename T, int ND, int P, bool VISC, bool DIAG>
__global__ void __launch_bounds__(256, 2) fused_jvp_kernel(FusedArgs<T> a, int epb) {
  using Sh = Shape<ND, P>;
  using Sm = FusedSmem<ND, P, VISC>;
  using S = Dual<T>;
  constexpr int NV = Sh::NV, NF = Sh::NF, NSP = Sh::NSP, NFP = Sh::NFP;
  constexpr int CT = Sm::CT, TB = Sm::TB, FO = Sm::FO;
  constexpr int NFPT = NF * NFP, ITERS = (NFPT + NSP - 1) / NSP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (gate_closed(a.gate)) return;
  const int le = threadIdx.x / NSP, lt = threadIdx.x % NSP;
  const int64_t i = (int64_t)blockIdx.x * epb + le;
  const bool valid = le < epb && i < a.count;
  T* base = reinterpret_cast<T*>(smem_raw) + (int64_t)le * Sm::PER;
  T* sqq = base;                 // [NV][NSP] own q
  T* sqv = sqq + NV * NSP;       // [NV][NSP] own v
  T* Aq = sqv + NV * NSP;        // [NF][CT][NFP] own compact traces of q
  T* Av = Aq + TB;               //                of v
  T* Bq = Av + TB;               // [NF][CT][NFP] the neighbour's traces of the shared face (its point order)
  T* Bv = Bq + TB;
  T* C = Aq + Sm::REG;           // [NF][FO / NFP][NFP] tangent F~com (then, NS: primal dq, tangent dq)
  S* sF = reinterpret_cast<S*>(Aq);   // [ND][NV][NSP] volume fluxes, once the faces are done
  const BasisTab<T>& B = a.basis[P];
  const int64_t slot = a.slot_begin + i;

  // 1. own state and tangent
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int64_t k = a.state_base + (i * NV + v) * NSP + lt;
      sqq[v * NSP + lt] = a.q[k];
      sqv[v * NSP + lt] = a.v[k];
    }
  }
  __syncthreads();

  // 2. own compact traces; the neighbours' traces of the shared faces
  if (valid) {
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
      const int fp = lt + it * NSP;
      if (fp >= NFPT) break;
      const int f = fp / NFP, t = fp % NFP;
      T qf[NV], dn[NV];
      trace_point<T, ND, P, VISC>(sqq, B, fp, qf, dn);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Aq[(f * CT + v) * NFP + t] = qf[v];
        if (VISC) Aq[(f * CT + NV + v) * NFP + t] = dn[v];
      }
      trace_point<T, ND, P, VISC>(sqv, B, fp, qf, dn);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Av[(f * CT + v) * NFP + t] = qf[v];
        if (VISC) Av[(f * CT + NV + v) * NFP + t] = dn[v];
      }
    }
    for (int idx = lt; idx < TB; idx += NSP) {
      const int f = idx / (CT * NFP), rem = idx % (CT * NFP);
      const FusedNbr nb = a.nbr[slot * NF + f];
      const int64_t src = a.ctrace_base + ((int64_t)nb.nloc * NF + nb.g) * CT * NFP + rem;
      Bq[idx] = a.trq[src];
      Bv[idx] = a.trv[src];
    }
  }
  __syncthreads();

  // 3. common flux, BR2 gradient and lifting at every face point of the element
  if (valid) {
    const int64_t e = a.slot_elem[slot];
#pragma unroll 1
    for (int it = 0; it < ITERS; ++it) {
      const int fp = lt + it * NSP;
      if (fp >= NFPT) break;
      const int f = fp / NFP, t = fp % NFP;
      const FusedNbr nb = a.nbr[slot * NF + f];
      const int u = orient_map(nb.code & 0xff, t, P, ND);
      const bool master = (nb.code >> 8) & 1;
      const int64_t eM = master ? e : (int64_t)nb.nelem, eS = master ? (int64_t)nb.nelem : e;
      const int fM = master ? f : nb.g, fS = master ? nb.g : f;
      const int tM = master ? t : u, tS = master ? u : t;
      const T* XqM = (master ? Aq : Bq) + f * CT * NFP;
      const T* XvM = (master ? Av : Bv) + f * CT * NFP;
      const T* XqS = (master ? Bq : Aq) + f * CT * NFP;
      const T* XvS = (master ? Bv : Av) + f * CT * NFP;
      S qM[NV], qS[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        qM[v] = S{XqM[v * NFP + tM], XvM[v * NFP + tM]};
        qS[v] = S{XqS[v * NFP + tS], XvS[v * NFP + tS]};
      }
      const int dm = fM >> 1, sm = fM & 1, ss = fS & 1;
      const T sgm = sm ? T(1) : T(-1);
      const T absA = geo_face(a.geo, eM, fM, ND * ND + 2 + dm, tM);
      const T inv_absA = geo_face(a.geo, eM, fM, ND * ND + 2 + ND + dm, tM);
      T A[ND], n[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        A[j] = sgm * geo_face(a.geo, eM, fM, dm * ND + j, tM);
        n[j] = A[j] * inv_absA;
      }
      S Fn[NV];
      common_flux<ND>(a.flux, qM, qS, n, absA, a.gamma, Fn);
      S qc[NV];
      if (VISC) {
#pragma unroll
        for (int v = 0; v < NV; ++v) qc[v] = T(0.5) * (qM[v] + qS[v]);
        const int ds = fS >> 1;
        T cM[ND], cS[ND];
        const T gJM = B.dgf[sm] * geo_face(a.geo, eM, fM, ND * ND + 1, tM);
        const T gJS = B.dgf[ss] * geo_face(a.geo, eS, fS, ND * ND + 1, tS);
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          cM[j] = gJM * geo_face(a.geo, eM, fM, dm * ND + j, tM);
          cS[j] = gJS * geo_face(a.geo, eS, fS, ds * ND + j, tS);
        }
        S GM[ND][NV], GS[ND][NV], Gc[ND][NV];
        face_grad<T, ND, P, DIAG>(XqM, XvM, fM, tM, a.geo, eM, B, GM);
        face_grad<T, ND, P, DIAG>(XqS, XvS, fS, tS, a.geo, eS, B, GS);
        if (DIAG) {
#pragma unroll
          for (int j = 0; j < ND; ++j)
#pragma unroll
            for (int v = 0; v < NV; ++v) Gc[j][v] = T(0.5) * (GM[j][v] + GS[j][v]);
#pragma unroll
          for (int j = 0; j < ND; ++j) {
            if (j != dm) continue;
#pragma unroll
            for (int v = 0; v < NV; ++v)
              Gc[j][v] = Gc[j][v] + T(0.5) * (cM[j] * (qc[v] - qM[v]) + cS[j] * (qc[v] - qS[v]));
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
      const T sgs = ss ? T(1) : T(-1);
      T* Cf = C + f * FO;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const S x = master ? sgm * Fn[v] : sgs * (T(0) - Fn[v]);
        Cf[v * NFP + t] = tangent(x);
        if (VISC) {
          const S dq = qc[v] - (master ? qM[v] : qS[v]);
          Cf[(NV + v) * NFP + t] = value(dq);
          Cf[(2 * NV + v) * NFP + t] = tangent(dq);
        }
      }
    }
  }
  __syncthreads();

  // 4. corrected gradient, fluxes, divergence and correction (as the volume kernel)
  int idx[3];
  idx[0] = lt % P;
  idx[1] = (lt / P) % P;
  idx[2] = ND == 3 ? lt / (P * P) : 0;
  T Smt[ND][ND];
  T Jinv = T(1);
  if (valid) {
    const int64_t e = a.slot_elem[slot];
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int j = 0; j < ND; ++j) Smt[d][j] = (DIAG && d != j) ? T(0) : geo_vol(a.geo, e, d * ND + j, lt);
    Jinv = geo_vol(a.geo, e, ND * ND + 1, lt);
    S q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = S{sqq[v * NSP + lt], sqv[v * NSP + lt]};
    S f[ND][NV];
    flux_inviscid<ND>(q, a.gamma, f);
    if (VISC) {
      S gref[ND][NV];
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
        const int lb = lt - idx[d] * stride;
        const int tf = face_pt<ND, P>(d, idx);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          Acc<S> acc = acc_init(szero<S>());
#pragma unroll
          for (int k = 0; k < P; ++k)
            acc_madd(acc, B.D[idx[d]][k], S{sqq[v * NSP + lb + k * stride], sqv[v * NSP + lb + k * stride]});
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const T* Cf = C + (2 * d + s) * FO;
            acc_madd(acc, B.dg[s][idx[d]], S{Cf[(NV + v) * NFP + tf], Cf[(2 * NV + v) * NFP + tf]});
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
            G[j][v] = (Smt[j][j] * Jinv) * gref[j][v];
          } else {
            S acc = szero<S>();
#pragma unroll
            for (int d = 0; d < ND; ++d) acc = acc + Smt[d][j] * gref[d][v];
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
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (DIAG) {
          sF[(d * NV + v) * NSP + lt] = Smt[d][d] * f[d][v];
        } else {
          S acc = szero<S>();
#pragma unroll
          for (int j = 0; j < ND; ++j) acc = acc + Smt[d][j] * f[j][v];
          sF[(d * NV + v) * NSP + lt] = acc;
        }
      }
  }
  __syncthreads();
  if (!valid) return;
  S div[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) div[v] = szero<S>();
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
    const int lb = lt - idx[d] * stride;
    const int tf = face_pt<ND, P>(d, idx);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const S* line = sF + (d * NV + v) * NSP + lb;
      Acc<S> acc = acc_init(szero<S>());
#pragma unroll
      for (int k = 0; k < P; ++k) acc_madd(acc, B.Dh[idx[d]][k], line[k * stride]);
#pragma unroll
      for (int s = 0; s < 2; ++s) acc_madd(acc, B.dg[s][idx[d]], S{T(0), C[(2 * d + s) * FO + v * NFP + tf]});
      div[v] = div[v] + acc_value(acc);
    }
  }
  const double vs = a.vscale ? *a.vscale : 1.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const S r = (T(0) - div[v]) * Jinv;
    const int64_t k = a.state_base + (i * NV + v) * NSP + lt;
    if (a.out_neg64) a.out_neg64[k] = -vs * (double)tangent(r);
    else a.out[k] = a.vscale ? (T)vs * tangent(r) : tangent(r);
  }
}

}  // namespace frgb

namespace frgb {

// ---------------------------------------------------------------------------
// Compact three-pass JVP (meshes whose faces are all interior and conforming):
// compact traces, then this face kernel, then the ordinary volume kernel.  A
// CTA takes FB faces of one group; both sides' compact traces of q and of v
// (4 blocks of CT x NFP values a face) are staged in shared memory, each
// thread forms both sides' physical gradients at its face point from them
// (face_grad: the stored normal derivative, the tangential ones differentiate
// the face trace) and evaluates the common flux, the BR2 gradient and the
// lifting once per face, writing the face outputs of both sides as the
// trace-gradient face kernel does.  Against that kernel the traces move 2 NV
// instead of NV (1 + ND) values a face point.
// ---------------------------------------------------------------------------
template <typename T>
struct CFaceArgs {
  const FaceRec* recs;
  const T* trq;             // compact traces of q and v
  const T* trv;
  T* fout;
  const BasisTab<T>* basis;
  GeoView<T> geo;
  T gamma, mu, kappa;
  int flux;
  int n;                    // faces in the group
  int nvt;                  // components of the trace-gradient layout (its offsets scale to compact ones)
  const int* gate = nullptr;   // see gate_closed
  // the tangent's traces formed in the face kernel (cface_vt_kernel): v in the
  // bucketed state layout and the group's bucket bases, which map a face
  // record's trace offset to its element's state block
  const T* v = nullptr;
  int64_t state_base = 0, trace_base = 0, ctrace_base = 0;
};

// Geometry of one face point read ahead of the staged traces (the master's
// area vector and |S|, both sides' metric terms for their gradients).
template <typename T, int ND>
struct CFaceGeo {
  T absA, inv_absA, JiM, JiS;
  T SfM[ND][ND], SfS[ND][ND];
  T rowM[ND], rowS[ND];
  int u;
};

template <typename T, int ND, int P, bool DIAG>
__device__ __forceinline__ void cface_geo(const CFaceArgs<T>& a, const FaceRec& r, int t, CFaceGeo<T, ND>& g) {
  const int dm = r.mf >> 1, ds = r.sf >> 1;
  g.u = orient_map(r.orient, t, P, ND);
  g.absA = geo_face(a.geo, r.me, r.mf, ND * ND + 2 + dm, t);
  g.inv_absA = geo_face(a.geo, r.me, r.mf, ND * ND + 2 + ND + dm, t);
  face_metric<T, ND, P, DIAG>(a.geo, r.me, r.mf, t, g.SfM, g.JiM);
  face_metric<T, ND, P, DIAG>(a.geo, r.se, r.sf, g.u, g.SfS, g.JiS);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    g.rowM[j] = geo_face(a.geo, r.me, r.mf, dm * ND + j, t);
    g.rowS[j] = geo_face(a.geo, r.se, r.sf, ds * ND + j, g.u);
  }
}

// Common flux, BR2 gradient and lifting at point t of one face from its four
// staged compact blocks (master q, master v, slave q, slave v), written as the
// face outputs of both sides.
template <typename T, int ND, int P, bool VISC, bool DIAG>
__device__ __forceinline__ void cface_point(const CFaceArgs<T>& a, const FaceRec& r, int t, const CFaceGeo<T, ND>& g,
                                            const T* XqM, const T* XvM, const T* XqS, const T* XvS) {
  using S = Dual<T>;
  constexpr int NV = ND + 2;
  constexpr int NFP = ND == 2 ? P : P * P;
  const BasisTab<T>& B = a.basis[P];
  const int dm = r.mf >> 1, sm = r.mf & 1, ss = r.sf & 1;
  const int u = g.u;
  S qM[NV], qS[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    qM[v] = S{XqM[v * NFP + t], XvM[v * NFP + t]};
    qS[v] = S{XqS[v * NFP + u], XvS[v * NFP + u]};
  }
  const T sgm = sm ? T(1) : T(-1);
  T A[ND], n[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    A[j] = sgm * g.rowM[j];
    n[j] = A[j] * g.inv_absA;
  }
  S Fn[NV];
  common_flux<ND>(a.flux, qM, qS, n, g.absA, a.gamma, Fn);
  S qc[NV];
  if (VISC) {
#pragma unroll
    for (int v = 0; v < NV; ++v) qc[v] = T(0.5) * (qM[v] + qS[v]);
    T cM[ND], cS[ND];
    const T gJM = B.dgf[sm] * g.JiM;
    const T gJS = B.dgf[ss] * g.JiS;
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      cM[j] = gJM * g.rowM[j];
      cS[j] = gJS * g.rowS[j];
    }
    S GM[ND][NV], GS[ND][NV], Gc[ND][NV];
    face_grad_m<T, ND, P, DIAG>(XqM, XvM, r.mf, t, g.SfM, g.JiM, B, GM);
    face_grad_m<T, ND, P, DIAG>(XqS, XvS, r.sf, u, g.SfS, g.JiS, B, GS);
    if (DIAG) {
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) Gc[j][v] = T(0.5) * (GM[j][v] + GS[j][v]);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        if (j != dm) continue;
#pragma unroll
        for (int v = 0; v < NV; ++v)
          Gc[j][v] = Gc[j][v] + T(0.5) * (cM[j] * (qc[v] - qM[v]) + cS[j] * (qc[v] - qS[v]));
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
  T* om = a.fout + r.mo;
  T* os = a.fout + r.so;
  const T sgs = ss ? T(1) : T(-1);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    om[v * NFP + t] = tangent(sgm * Fn[v]);
    os[v * NFP + u] = tangent(sgs * (T(0) - Fn[v]));
    if (VISC) {
      const S dM = qc[v] - qM[v], dS = qc[v] - qS[v];
      om[(NV + v) * NFP + t] = value(dM);
      om[(2 * NV + v) * NFP + t] = tangent(dM);
      os[(NV + v) * NFP + u] = value(dS);
      os[(2 * NV + v) * NFP + u] = tangent(dS);
    }
  }
}

template <typename T, int ND, int P, bool VISC, bool DIAG>
__global__ void __launch_bounds__(128, 4) cface_kernel(CFaceArgs<T> a) {
  constexpr int NV = ND + 2;
  constexpr int NFP = ND == 2 ? P : P * P;
  constexpr int CT = CompactWidth<VISC, NV>::value;
  constexpr int FB = NFP >= 128 ? 1 : 128 / NFP;    // faces a CTA
  constexpr int BLK = CT * NFP;
  __shared__ T sh[FB][4][BLK];                        // master q, master v, slave q, slave v
  if (gate_closed(a.gate)) return;
  const int lf = threadIdx.x / NFP, t = threadIdx.x % NFP;
  const int64_t fidx = (int64_t)blockIdx.x * FB + lf;
  const bool valid = lf < FB && fidx < a.n;
  FaceRec r{};
  CFaceGeo<T, ND> g{};
  if (valid) {
    r = a.recs[fidx];
    // compact trace blocks of the two sides: on a conforming mesh the compact
    // offset is the trace-gradient one scaled by CT / nvt
    const int64_t om = r.mt / a.nvt * CT, osl = r.st / a.nvt * CT;
    T buf[4][CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      buf[0][c] = a.trq[om + c * NFP + t];
      buf[1][c] = a.trv[om + c * NFP + t];
      buf[2][c] = a.trq[osl + c * NFP + t];
      buf[3][c] = a.trv[osl + c * NFP + t];
    }
    cface_geo<T, ND, P, DIAG>(a, r, t, g);
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int c = 0; c < CT; ++c) sh[lf][w][c * NFP + t] = buf[w][c];
  }
  __syncthreads();
  if (!valid) return;
  cface_point<T, ND, P, VISC, DIAG>(a, r, t, g, sh[lf][0], sh[lf][1], sh[lf][2], sh[lf][3]);
}

// ---------------------------------------------------------------------------
// The same face work with the staging done by the copy engine: a persistent
// CTA walks the groups' face tiles; for each tile one lane per face issues
// four bulk asynchronous copies (cp.async.bulk, global -> shared, completion
// counted in bytes on an mbarrier), one per compact block, and the copies of
// the next tile are in flight while the threads compute the current one (two
// buffers, one barrier a tile).  Blocks must be multiples of 16 bytes at
// 16-byte aligned offsets (the host checks CT x NFP x sizeof(T)); a wait that
// exceeds its iteration limit sets bit 0 of *status, stops the walk and waits,
// again bounded, for the copies still in flight before the CTA exits.
// Instantiated for FP32 only (two buffers within the 48 KB of static shared
// memory).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait: true when the phase of `parity` completed within `limit` tries
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

constexpr int kTmaWaitLimit = 1 << 22;   // tries of one wait before it gives up (far above any copy's latency)

template <typename T, int ND, int P, bool VISC, bool DIAG>
__global__ void __launch_bounds__(128, 4) cface_tma_kernel(CFaceArgs<T> a, int* status) {
  constexpr int NV = ND + 2;
  constexpr int NFP = ND == 2 ? P : P * P;
  constexpr int CT = CompactWidth<VISC, NV>::value;
  constexpr int FB = NFP >= 128 ? 1 : 128 / NFP;
  constexpr int BLK = CT * NFP;
  constexpr uint32_t BYTES = BLK * sizeof(T);
  static_assert(BYTES % 16 == 0 && FB <= 32, "bulk-copied blocks: multiples of 16 bytes, at most one warp of faces");
  __shared__ __align__(128) T sh[2][FB][4][BLK];
  __shared__ __align__(8) uint64_t bar[2];
  if (gate_closed(a.gate)) return;   // before any barrier is armed or copy issued
  const int lf = threadIdx.x / NFP, t = threadIdx.x % NFP;
  const int ntiles = (a.n + FB - 1) / FB;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // one lane per face of the tile issues its four copies after lane 0 has
  // announced the tile's bytes
  auto issue = [&](int tile, int b) {
    const int64_t f0 = (int64_t)tile * FB;
    const int nf = (int)min((int64_t)FB, (int64_t)a.n - f0);
    const int lane = threadIdx.x;   // warp 0
    if (lane == 0) mbar_arrive_expect(&bar[b], (uint32_t)nf * 4u * BYTES);
    __syncwarp();
    if (lane < nf) {
      const FaceRec r = a.recs[f0 + lane];
      const int64_t om = r.mt / a.nvt * CT, osl = r.st / a.nvt * CT;
      bulk_copy_g2s(sh[b][lane][0], a.trq + om, BYTES, &bar[b]);
      bulk_copy_g2s(sh[b][lane][1], a.trv + om, BYTES, &bar[b]);
      bulk_copy_g2s(sh[b][lane][2], a.trq + osl, BYTES, &bar[b]);
      bulk_copy_g2s(sh[b][lane][3], a.trv + osl, BYTES, &bar[b]);
    }
  };
  int it = 0;
  bool stop = false;
  if ((int)blockIdx.x < ntiles && threadIdx.x < 32) issue(blockIdx.x, 0);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    const int next = tile + gridDim.x;
    if (next < ntiles && threadIdx.x < 32) issue(next, b ^ 1);
    const int64_t fidx = (int64_t)tile * FB + lf;
    const bool valid = lf < FB && fidx < a.n;
    FaceRec r{};
    CFaceGeo<T, ND> g{};
    if (valid) {
      r = a.recs[fidx];
      cface_geo<T, ND, P, DIAG>(a, r, t, g);
    }
    // every thread waits for the tile's bytes itself; one barrier a tile then
    // frees buffer b for the tile after next and carries a timeout to the
    // whole CTA
    const bool ok = mbar_wait(&bar[b], (uint32_t)((it >> 1) & 1), kTmaWaitLimit);
    if (!ok) atomicOr(status, 1);
    if (ok && valid)
      cface_point<T, ND, P, VISC, DIAG>(a, r, t, g, sh[b][lf][0], sh[b][lf][1], sh[b][lf][2], sh[b][lf][3]);
    if (__syncthreads_or(!ok)) {
      stop = true;
      break;
    }
  }
  if (stop) {
    // copies of this and the next tile may still be in flight: wait for both
    // buffers' current phases, bounded, before the CTA's shared memory goes away
    mbar_wait(&bar[it & 1], (uint32_t)((it >> 1) & 1), kTmaWaitLimit);
    mbar_wait(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1), kTmaWaitLimit);
  }
}

// ---------------------------------------------------------------------------
// The compact face pass with the tangent's traces formed in the face kernel
// (two passes a product instead of three: no trace pass over v and no round
// trip of its compact traces through memory).  Per face of a tile, four
// blocks are copied into shared memory: the two sides' compact traces of q
// (fixed during a GMRES solve) and the two sides' elements of v ([NV][NSP],
// contiguous in the bucketed state).  Each thread forms the compact trace of
// v at its point of both faces (the interpolation of the trace pass, with the
// same explicit fused multiply-adds, so the values have the same bits), the
// face's threads meet at a warp barrier, and the flux step follows.  A face's
// points lie in one warp (32 a multiple of the face's points), so no CTA
// barrier separates the two steps.
//
// Buffers: the q-trace blocks are double-buffered and issued one tile ahead
// by warp 0, as in cface_tma_kernel; the element blocks, twice their size,
// have one buffer, and the last warp to finish forming its traces (a shared
// counter) issues the next tile's element copies, so that they overlap the
// flux step.  Both land on the next tile's barrier, which expects all of its
// bytes from the start.  One CTA barrier a tile frees the q-trace buffer and
// the tangent traces; the bounded waits and the error path are those of
// cface_tma_kernel.  Shared memory: 50 KB for 3D p = 3 (four CTAs an SM).
// ---------------------------------------------------------------------------
template <typename T, int ND, int P, bool VISC>
struct CFaceVt {
  static constexpr int NV = ND + 2;
  static constexpr int NFP = ND == 2 ? P : P * P;
  static constexpr int NSP = Shape<ND, P>::NSP;
  static constexpr int CT = CompactWidth<VISC, NV>::value;
  static constexpr int FB = 128 / NFP;                 // faces a tile
  static constexpr int NW = 4;                         // warps a CTA
  static constexpr int BLK = CT * NFP;                 // compact trace block of one face side
  static constexpr int EL = NV * NSP;                  // state block of one element
  static constexpr uint32_t QB = BLK * sizeof(T), EB = EL * sizeof(T);
  static constexpr bool OK = 32 % NFP == 0 && FB <= 32 && QB % 16 == 0 && EB % 16 == 0;
  // [2][FB][2][BLK] q traces, [FB][2][EL] elements of v, [FB][2][BLK] tangent traces
  static constexpr size_t Q_OFF = 0, E_OFF = (size_t)2 * FB * 2 * BLK, V_OFF = E_OFF + (size_t)FB * 2 * EL;
  static constexpr size_t SMEM = (V_OFF + (size_t)FB * 2 * BLK) * sizeof(T);
};

template <typename T, int ND, int P, bool VISC, bool DIAG>
__global__ void __launch_bounds__(128, 4) cface_vt_kernel(CFaceArgs<T> a, int* status) {
  using C = CFaceVt<T, ND, P, VISC>;
  constexpr int NV = C::NV, NFP = C::NFP, NF = 2 * ND, FB = C::FB, BLK = C::BLK, EL = C::EL;
  static_assert(C::OK, "a face's points within one warp; bulk-copied blocks multiples of 16 bytes");
  extern __shared__ __align__(16) unsigned char smem_raw[];   // bulk-copy destinations: 16-byte aligned
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t nidx[FB][2];    // the next tile's elements (bucket-local), for its element copies
  __shared__ int done;               // warps done forming the current tile's traces
  T* const sb = reinterpret_cast<T*>(smem_raw);
  if (gate_closed(a.gate)) return;   // before any barrier is armed or copy issued
  const int lf = threadIdx.x / NFP, t = threadIdx.x % NFP, lane = threadIdx.x & 31;
  const int ntiles = (a.n + FB - 1) / FB;
  const uint64_t per_elem = (uint64_t)a.nvt * NFP * NF;  // trace-gradient values of one element
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    done = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto faces_of = [&](int tile) { return (int)min((int64_t)FB, (int64_t)a.n - (int64_t)tile * FB); };
  // warp 0: announce the tile's bytes (both kinds), copy its q-trace blocks
  // into buffer b and leave its elements in nidx (one lane per face)
  auto issue_q = [&](int tile, int b) {
    const int nf = faces_of(tile);
    if (lane == 0) mbar_arrive_expect(&bar[b], (uint32_t)nf * 2u * (C::QB + C::EB));
    __syncwarp();
    if (lane < nf) {
      const FaceRec r = a.recs[(int64_t)tile * FB + lane];
      // the two sides' bucket-local elements (a 32-bit division while the
      // bucket's trace offsets fit), then their blocks
      const uint64_t rm = (uint64_t)(r.mt - a.trace_base), rs = (uint64_t)(r.st - a.trace_base);
      const int64_t im = rm >> 32 ? (int64_t)(rm / per_elem) : (int64_t)((uint32_t)rm / (uint32_t)per_elem);
      const int64_t is = rs >> 32 ? (int64_t)(rs / per_elem) : (int64_t)((uint32_t)rs / (uint32_t)per_elem);
      T* dst = sb + C::Q_OFF + (size_t)(b * FB + lane) * 2 * BLK;
      bulk_copy_g2s(dst, a.trq + a.ctrace_base + (im * NF + r.mf) * BLK, C::QB, &bar[b]);
      bulk_copy_g2s(dst + BLK, a.trq + a.ctrace_base + (is * NF + r.sf) * BLK, C::QB, &bar[b]);
      nidx[lane][0] = im;
      nidx[lane][1] = is;
    }
  };
  // one warp: copy the elements recorded in nidx into the element buffer
  auto issue_v = [&](int tile, int b) {
    const int nf = faces_of(tile);
    if (lane < nf) {
      T* dst = sb + C::E_OFF + (size_t)lane * 2 * EL;
      bulk_copy_g2s(dst, a.v + a.state_base + nidx[lane][0] * EL, C::EB, &bar[b]);
      bulk_copy_g2s(dst + EL, a.v + a.state_base + nidx[lane][1] * EL, C::EB, &bar[b]);
    }
  };
  const BasisTab<T>& B = a.basis[P];
  T* const xv = sb + C::V_OFF + (size_t)lf * 2 * BLK;
  int it = 0;
  bool stop = false;
  if ((int)blockIdx.x < ntiles && threadIdx.x < 32) {
    issue_q(blockIdx.x, 0);
    __syncwarp();
    issue_v(blockIdx.x, 0);
  }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    const int next = tile + gridDim.x;
    if (next < ntiles && threadIdx.x < 32) issue_q(next, b ^ 1);
    const int64_t fidx = (int64_t)tile * FB + lf;
    const bool valid = fidx < a.n;
    FaceRec r{};
    CFaceGeo<T, ND> g{};
    if (valid) {
      r = a.recs[fidx];
      cface_geo<T, ND, P, DIAG>(a, r, t, g);
    }
    // every thread waits for the tile's bytes itself (see cface_tma_kernel)
    const bool ok = mbar_wait(&bar[b], (uint32_t)((it >> 1) & 1), kTmaWaitLimit);
    if (!ok) atomicOr(status, 1);
    if (ok && valid) {
      // the tangent's compact trace at this thread's point of the master face
      // and at the same-numbered point of the slave face (slave numbering)
      const T* el = sb + C::E_OFF + (size_t)lf * 2 * EL;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        T qf[NV], dn[NV];
        trace_point<T, ND, P, VISC, line_vec_width<T, P, C::NSP, BLK>() < line_vec_width<T, P, C::NSP, EL>()
                                         ? line_vec_width<T, P, C::NSP, BLK>()
                                         : line_vec_width<T, P, C::NSP, EL>()>(
            el + side * EL, B, (side ? r.sf : r.mf) * NFP + t, qf, dn);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          xv[side * BLK + v * NFP + t] = qf[v];
          if (VISC) xv[side * BLK + (NV + v) * NFP + t] = dn[v];
        }
      }
    }
    // the face's points are this warp's lanes: its traces are complete here;
    // the CTA barrier at the end of the previous tile ordered these writes
    // after every read of the last tile's traces
    __syncwarp();
    // this warp is done with the element buffer: the last warp to get here
    // refills it with the next tile's elements (the fences order the other
    // warps' reads of the buffer and warp 0's nidx before the copies)
    int last = 0;
    if (lane == 0) {
      __threadfence_block();
      last = atomicAdd(&done, 1) == C::NW - 1;
      if (last) {
        done = 0;   // the next tile's arrivals follow the CTA barrier below
        __threadfence_block();
      }
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    __syncwarp();   // the lanes' nidx reads follow lane 0's fence
    if (last && ok && next < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_v(next, b ^ 1);
    }
    if (ok && valid) cface_point<T, ND, P, VISC, DIAG>(a, r, t, g, sb + C::Q_OFF + (size_t)(b * FB + lf) * 2 * BLK,
                                                        xv, sb + C::Q_OFF + (size_t)(b * FB + lf) * 2 * BLK + BLK,
                                                        xv + BLK);
    if (__syncthreads_or(!ok)) {
      stop = true;
      break;
    }
  }
  if (stop) {
    // copies of this and the next tile may still be in flight: wait for both
    // buffers' current phases, bounded, before the CTA's shared memory goes away
    mbar_wait(&bar[it & 1], (uint32_t)((it >> 1) & 1), kTmaWaitLimit);
    mbar_wait(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1), kTmaWaitLimit);
  }
}

}  // namespace frgb

