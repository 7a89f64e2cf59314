// Adjoint (VJP) kernels of the FR residual: the exact transpose of the
// linearisation that fr_jvp evaluates, in reverse order of the forward passes
//   trace -> face -> volume     becomes     volume^T -> face^T -> trace^T.
// Every adjoint value is written by exactly one thread into a slot it owns
// (element-face blocks), and gathered by the consumer: no floating-point
// atomics, so the result is deterministic.
//
// Buffers: fbar has the layout of fout (comp 0..NV-1: adjoint of F~^com,
// NV..2NV-1: adjoint of dq = q^com - q); trbar has the layout of the traces
// (comp 0..NV-1: adjoint of the q trace; NV + d*NV + v: adjoint of the
// reference derivative d_xi_d q_v at the face point).
#pragma once

#include "fr_kernels.cuh"

namespace frgb {

// Transpose of the linear map G -> f_v(q, G) at fixed q: Gb = (d f_v / d G)^T fb.
template <int ND, typename T>
__device__ __forceinline__ void viscous_adjoint_G(const T* q, const T (*fb)[ND + 2], T gamma, T mu,
                                                  T kappa, T (*Gb)[ND + 2]) {
  constexpr int NV = ND + 2;
  const T rinv = T(1) / q[0];
  T vel[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) vel[i] = q[1 + i] * rinv;
  const T Es = q[NV - 1] * rinv;
  T taub[ND][ND], dub[ND][ND], dTb[ND], dEb[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) taub[i][j] = fb[j][1 + i] + vel[i] * fb[j][NV - 1];
#pragma unroll
  for (int j = 0; j < ND; ++j) dTb[j] = kappa * fb[j][NV - 1];
  T trace_tb = T(0);
#pragma unroll
  for (int i = 0; i < ND; ++i) trace_tb += taub[i][i];
  const T divb = -T(2.0 / 3.0) * mu * trace_tb;
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) dub[i][j] = mu * (taub[i][j] + taub[j][i]) + (i == j ? divb : T(0));
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    dEb[j] = (gamma - T(1)) * dTb[j];
#pragma unroll
    for (int k = 0; k < ND; ++k) dub[k][j] -= (gamma - T(1)) * vel[k] * dTb[j];
  }
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    T g0 = -Es * dEb[j];
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      Gb[j][1 + i] = dub[i][j] * rinv;
      g0 -= vel[i] * dub[i][j];
    }
    Gb[j][0] = g0 * rinv;
    Gb[j][NV - 1] = dEb[j] * rinv;
  }
}

// qb += (d/dq [f_inv(q)*si - f_v(q, G)*sv])^T fb by NV forward-mode sweeps.
template <int ND, typename T>
__device__ __forceinline__ void flux_adjoint_q(const T* q, const T (*G)[ND + 2], const T (*fb)[ND + 2],
                                               T gamma, T mu, T kappa, bool inv, bool visc, T* qb) {
  constexpr int NV = ND + 2;
  using D = Dual<T>;
#pragma unroll 1
  for (int k = 0; k < NV; ++k) {
    D qd[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) qd[v] = D{q[v], v == k ? T(1) : T(0)};
    T acc = T(0);
    if (inv) {
      D f[ND][NV];
      flux_inviscid<ND>(qd, gamma, f);
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc += fb[j][v] * f[j][v].d;
    }
    if (visc) {
      D Gd[ND][NV], fv[ND][NV];
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) Gd[j][v] = D{G[j][v], T(0)};
      flux_viscous<ND>(qd, Gd, gamma, mu, kappa, fv);
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc -= fb[j][v] * fv[j][v].d;
    }
    qb[k] += acc;
  }
}

// (qLb, qRb) += (d Fn / d(qL, qR))^T Fnb for the common flux of kind `kind`
// (Rusanov or Roe, area included): one forward-mode column per input.
template <int ND, typename T>
__device__ __forceinline__ void flux_adjoint(int kind, const T* qL, const T* qR, const T* n, T absA, T gamma,
                                             const T* Fnb, T* qLb, T* qRb) {
  constexpr int NV = ND + 2;
  using D = Dual<T>;
#pragma unroll 1
  for (int k = 0; k < 2 * NV; ++k) {
    D a[NV], b[NV], Fn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      a[v] = D{qL[v], k == v ? T(1) : T(0)};
      b[v] = D{qR[v], k == NV + v ? T(1) : T(0)};
    }
    common_flux<ND>(kind, a, b, n, absA, gamma, Fn);
    T acc = T(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc += Fnb[v] * Fn[v].d;
    if (k < NV) qLb[k] += acc; else qRb[k - NV] += acc;
  }
}

// ---------------------------------------------------------------------------
// Volume adjoint.  One thread per solution point, EPB elements per block.
// ---------------------------------------------------------------------------
template <typename T>
struct VolAdjArgs {
  const T* q;
  const T* w;
  T* out;              // partial q-bar (volume terms)
  const T* fout;       // forward face outputs (primal dq)
  T* fbar;             // adjoints of F~^com and dq
  const int32_t* slot_elem;
  const BasisTab<T>* basis;
  GeoView<T> geo;
  T gamma, mu, kappa;
  int64_t state_base, out_base;
  int count, slot_begin;
};

template <typename T, int ND, int P, bool VISC>
__global__ void __launch_bounds__(VolCfg<ND, P>::THREADS) vol_adj_kernel(VolAdjArgs<T> a) {
  using Sh = Shape<ND, P>;
  constexpr int NV = Sh::NV, NF = Sh::NF, NSP = Sh::NSP, NFP = Sh::NFP;
  constexpr int EPB = VolCfg<ND, P>::EPB;
  constexpr int FS = 3 * NV * NFP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int le = threadIdx.x / NSP;
  const int sp = threadIdx.x % NSP;
  const int64_t i = (int64_t)blockIdx.x * EPB + le;
  const bool valid = i < a.count;
  T* sq = sm + le * (2 * NV + 2 * ND * NV) * NSP;   // [NV][NSP]
  T* sdb = sq + NV * NSP;                            // div-bar [NV][NSP]
  T* sFb = sdb + NV * NSP;                           // [ND][NV][NSP] unused slot kept for alignment
  T* sgb = sFb + ND * NV * NSP;                      // gref-bar [ND][NV][NSP]
  const BasisTab<T>& B = a.basis[P];
  int idx[3];
  idx[0] = sp % P;
  idx[1] = (sp / P) % P;
  idx[2] = ND == 3 ? sp / (P * P) : 0;
  const int64_t e = valid ? a.slot_elem[a.slot_begin + i] : 0;
  const T* fo = a.fout + (valid ? a.out_base + i * NF * FS : 0);
  T* fb = a.fbar + (valid ? a.out_base + i * NF * FS : 0);

  T q[NV];
  T Sm[ND][ND];
  T Jinv = T(1);
  if (valid) {
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int j = 0; j < ND; ++j) Sm[d][j] = geo_vol(a.geo, e, d * ND + j, sp);
    Jinv = geo_vol(a.geo, e, ND * ND + 1, sp);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      q[v] = a.q[a.state_base + (i * NV + v) * NSP + sp];
      sq[v * NSP + sp] = q[v];
      sdb[v * NSP + sp] = -a.w[a.state_base + (i * NV + v) * NSP + sp] * Jinv;
    }
  }
  __syncthreads();

  T qb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) qb[v] = T(0);
  if (valid) {
    // F~-bar_d at this point and the adjoint of F~^com on the faces
    T Fb[ND][NV];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
      const int base = sp - idx[d] * stride;
      const int tf = face_pt<ND, P>(d, idx);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T* line = sdb + v * NSP + base;
        T acc = T(0), gl[2] = {T(0), T(0)};
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const T x = line[k * stride];
          acc += B.D[k][idx[d]] * x;
          gl[0] += B.dg[0][k] * x;
          gl[1] += B.dg[1][k] * x;
        }
        acc -= B.ext[0][idx[d]] * gl[0] + B.ext[1][idx[d]] * gl[1];
        Fb[d][v] = acc;
        if (idx[d] == 0) {
          fb[(2 * d + 0) * FS + v * NFP + tf] = gl[0];
          fb[(2 * d + 1) * FS + v * NFP + tf] = gl[1];
        }
      }
    }
    T fbar[ND][NV];
#pragma unroll
    for (int j = 0; j < ND; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T acc = T(0);
#pragma unroll
        for (int d = 0; d < ND; ++d) acc += Sm[d][j] * Fb[d][v];
        fbar[j][v] = acc;
      }
    T G[ND][NV];
    if (VISC) {
      T gref[ND][NV];
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
        const int base = sp - idx[d] * stride;
        const int tf = face_pt<ND, P>(d, idx);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T acc = T(0);
#pragma unroll
          for (int k = 0; k < P; ++k) acc += B.D[idx[d]][k] * sq[v * NSP + base + k * stride];
#pragma unroll
          for (int s = 0; s < 2; ++s) acc += B.dg[s][idx[d]] * fo[(2 * d + s) * FS + (NV + v) * NFP + tf];
          gref[d][v] = acc;
        }
      }
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T acc = T(0);
#pragma unroll
          for (int d = 0; d < ND; ++d) acc += Sm[d][j] * gref[d][v];
          G[j][v] = acc * Jinv;
        }
    }
    flux_adjoint_q<ND>(q, G, fbar, a.gamma, a.mu, a.kappa, true, VISC, qb);
    if (VISC) {
      T Gb[ND][NV], negf[ND][NV];
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) negf[j][v] = -fbar[j][v];
      viscous_adjoint_G<ND>(q, negf, a.gamma, a.mu, a.kappa, Gb);
#pragma unroll
      for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T acc = T(0);
#pragma unroll
          for (int j = 0; j < ND; ++j) acc += Sm[d][j] * Gb[j][v];
          sgb[(d * NV + v) * NSP + sp] = acc * Jinv;
        }
    }
  }
  if (VISC) __syncthreads();
  if (!valid) return;
  if (VISC) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
      const int base = sp - idx[d] * stride;
      const int tf = face_pt<ND, P>(d, idx);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T* line = sgb + (d * NV + v) * NSP + base;
        T acc = T(0), gl[2] = {T(0), T(0)};
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const T x = line[k * stride];
          acc += B.D[k][idx[d]] * x;
          gl[0] += B.dg[0][k] * x;
          gl[1] += B.dg[1][k] * x;
        }
        qb[v] += acc;
        if (idx[d] == 0) {
          fb[(2 * d + 0) * FS + (NV + v) * NFP + tf] = gl[0];
          fb[(2 * d + 1) * FS + (NV + v) * NFP + tf] = gl[1];
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) a.out[a.state_base + (i * NV + v) * NSP + sp] = qb[v];
}

// ---------------------------------------------------------------------------
// Face adjoint (interior).  One thread per (face, mortar point).
// ---------------------------------------------------------------------------
template <typename T>
struct FaceAdjArgs {
  const FaceRec* recs;
  const T* trq;        // primal traces
  const T* fbar;       // adjoints of the face outputs
  T* trbar;            // adjoints of the traces
  T* scratch;          // mixed groups: slave adjoints on the mortar (master order)
  const BasisTab<T>* basis;
  const MortarTab<T>* mortar;
  GeoView<T> geo_m, geo_s;
  T gamma, mu, kappa;
  int n, Pm, Ps;
  int flux;            // common inviscid flux: 0 Rusanov, 1 Roe
  int64_t scratch_base;
};

// reference-derivative adjoint from the physical-gradient adjoint at a face point
template <int ND, typename T>
__device__ __forceinline__ void gradient_to_ref_adjoint(const GeoView<T>& g, int64_t e, int f, int t,
                                                        const T (*Gb)[ND + 2], T (*dqb)[ND + 2]) {
  constexpr int NV = ND + 2;
  const T Jinv = geo_face(g, e, f, ND * ND + 1, t);
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < ND; ++j) acc += geo_face(g, e, f, d * ND + j, t) * Gb[j][v];
      dqb[d][v] = acc * Jinv;
    }
}

template <typename T, int ND, bool VISC>
__global__ void __launch_bounds__(128) face_adj_kernel(FaceAdjArgs<T> a) {
  constexpr int NV = ND + 2;
  const int Pm = a.Pm, Ps = a.Ps;
  const int NFPm = ND == 2 ? Pm : Pm * Pm;
  const int NFPs = ND == 2 ? Ps : Ps * Ps;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)a.n * NFPm) return;
  const int t = (int)(gid % NFPm);
  const FaceRec r = a.recs[gid / NFPm];
  const int dm = r.mf >> 1, sm = r.mf & 1, ss = r.sf & 1;
  const int u = orient_map(r.orient, t, Pm, ND);
  const bool conf = Pm == Ps;
  const int ua = u % Pm, ub = ND == 2 ? 0 : u / Pm;

  // primal values on the mortar
  T qM[NV], qS[NV];
  FaceArgs<T> fa{};
  fa.trq = a.trq;
  fa.trv = nullptr;
  fa.Pm = Pm;
  fa.Ps = Ps;
  fa.mortar = a.mortar;
  load_trace_pt<ND>(a.trq, (const T*)nullptr, r.mt, 0, NV, NFPm, t, qM);
  slave_at_mortar<ND>(fa, r.st, 0, NV, u, qS);
  T A[ND], n[ND];
  const T sgm = sm ? T(1) : T(-1), sgs = ss ? T(1) : T(-1);
  const T absA = geo_face(a.geo_m, r.me, r.mf, ND * ND + 2 + dm, t);
  const T inv_absA = geo_face(a.geo_m, r.me, r.mf, ND * ND + 2 + ND + dm, t);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    A[j] = sgm * geo_face(a.geo_m, r.me, r.mf, dm * ND + j, t);
    n[j] = A[j] * inv_absA;
  }

  // adjoint seeds
  T Fnb[NV], qcb[NV], qMb[NV], qSb[NV];
  const T* fbm = a.fbar + r.mo;
  const T* fbs = a.fbar + r.so;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Fnb[v] = sgm * fbm[v * NFPm + t];
    qcb[v] = VISC ? fbm[(NV + v) * NFPm + t] : T(0);
    qMb[v] = VISC ? -fbm[(NV + v) * NFPm + t] : T(0);
    qSb[v] = T(0);
  }
  if (conf) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Fnb[v] -= sgs * fbs[v * NFPs + u];
      if (VISC) {
        qcb[v] += fbs[(NV + v) * NFPs + u];
        qSb[v] -= fbs[(NV + v) * NFPs + u];
      }
    }
  } else {
    // transpose of the L2 projection onto the slave side
    for (int pb = 0; pb < (ND == 2 ? 1 : Ps); ++pb) {
      const T wb = ND == 2 ? T(1) : a.mortar->Pi[pb][ub];
      for (int pa = 0; pa < Ps; ++pa) {
        const T w = a.mortar->Pi[pa][ua] * wb;
        const int pt = pa + Ps * pb;
        for (int v = 0; v < NV; ++v) {
          Fnb[v] -= sgs * w * fbs[v * NFPs + pt];
          if (VISC) qcb[v] += w * fbs[(NV + v) * NFPs + pt];
        }
      }
    }
  }
  flux_adjoint<ND>(a.flux, qM, qS, n, absA, a.gamma, Fnb, qMb, qSb);
  T GMb[ND][NV], GSb[ND][NV];
  if (VISC) {
    T qc[NV], cM[ND], cS[ND];
#pragma unroll
    for (int v = 0; v < NV; ++v) qc[v] = T(0.5) * (qM[v] + qS[v]);
    const T gJ = a.basis[Pm].dgf[sm] * geo_face(a.geo_m, r.me, r.mf, ND * ND + 1, t);
#pragma unroll
    for (int j = 0; j < ND; ++j) cM[j] = gJ * geo_face(a.geo_m, r.me, r.mf, dm * ND + j, t);
    {
      FaceArgs<T> fb2 = fa;
      fb2.basis = a.basis;
      fb2.geo_s = a.geo_s;
      slave_coef_at_mortar<ND>(fb2, r, u, cS);
    }
    T GM[ND][NV], GS[ND][NV], Gc[ND][NV];
    load_trace_pt<ND>(a.trq, (const T*)nullptr, r.mt, NV, ND * NV, NFPm, t, &GM[0][0]);
    slave_at_mortar<ND>(fa, r.st, NV, ND * NV, u, &GS[0][0]);
#pragma unroll
    for (int j = 0; j < ND; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v)
        Gc[j][v] = T(0.5) * (GM[j][v] + cM[j] * (qc[v] - qM[v]) + GS[j][v] + cS[j] * (qc[v] - qS[v]));
    // Fn -= sum_j fv(qc, Gc)[j] A_j
    T fvb[ND][NV], Gcb[ND][NV];
#pragma unroll
    for (int j = 0; j < ND; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) fvb[j][v] = -Fnb[v] * A[j];
    viscous_adjoint_G<ND>(qc, fvb, a.gamma, a.mu, a.kappa, Gcb);
    // explicit qc dependence of fv: flux_adjoint_q with inv=false subtracts, so pass -fvb
    {
      T nfvb[ND][NV];
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) nfvb[j][v] = -fvb[j][v];
      flux_adjoint_q<ND>(qc, Gc, nfvb, a.gamma, a.mu, a.kappa, false, true, qcb);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T sM = T(0), sS = T(0);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        GMb[j][v] = T(0.5) * Gcb[j][v];
        GSb[j][v] = T(0.5) * Gcb[j][v];
        sM += cM[j] * Gcb[j][v];
        sS += cS[j] * Gcb[j][v];
      }
      qcb[v] += T(0.5) * (sM + sS);
      qMb[v] -= T(0.5) * sM;
      qSb[v] -= T(0.5) * sS;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      qMb[v] += T(0.5) * qcb[v];
      qSb[v] += T(0.5) * qcb[v];
    }
  }
  // master side: trace adjoints at its own point
  T* tm = a.trbar + r.mt;
#pragma unroll
  for (int v = 0; v < NV; ++v) tm[v * NFPm + t] = qMb[v];
  if (VISC) {
    T dqb[ND][NV];
    gradient_to_ref_adjoint<ND>(a.geo_m, r.me, r.mf, t, GMb, dqb);
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
      for (int v = 0; v < NV; ++v) tm[(NV + d * NV + v) * NFPm + t] = dqb[d][v];
  }
  if (conf) {
    T* ts = a.trbar + r.st;
#pragma unroll
    for (int v = 0; v < NV; ++v) ts[v * NFPs + u] = qSb[v];
    if (VISC) {
      T dqb[ND][NV];
      gradient_to_ref_adjoint<ND>(a.geo_s, r.se, r.sf, u, GSb, dqb);
#pragma unroll
      for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int v = 0; v < NV; ++v) ts[(NV + d * NV + v) * NFPs + u] = dqb[d][v];
    }
  } else {
    T* sc = a.scratch + a.scratch_base + (int64_t)r.idx * 4 * NV * NFPm;
#pragma unroll
    for (int v = 0; v < NV; ++v) sc[v * NFPm + t] = qSb[v];
    if (VISC) {
#pragma unroll
      for (int j = 0; j < ND; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) sc[(NV + j * NV + v) * NFPm + t] = GSb[j][v];
    }
  }
}

// Mixed faces: transpose of the slave interpolation to the mortar, plus the
// direct -dq-bar term.  One thread per (face, slave point).
template <typename T, int ND, bool VISC>
__global__ void __launch_bounds__(128) mortar_gather_adj_kernel(FaceAdjArgs<T> a) {
  constexpr int NV = ND + 2;
  const int Pm = a.Pm, Ps = a.Ps;
  const int NFPm = ND == 2 ? Pm : Pm * Pm;
  const int NFPs = ND == 2 ? Ps : Ps * Ps;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)a.n * NFPs) return;
  const int pt = (int)(gid % NFPs);
  const FaceRec r = a.recs[gid / NFPs];
  const int pa = pt % Ps, pb = ND == 2 ? 0 : pt / Ps;
  const T* sc = a.scratch + a.scratch_base + (int64_t)r.idx * 4 * NV * NFPm;
  constexpr int NC = VISC ? NV * (1 + ND) : NV;
  T acc[NV * (1 + ND)];
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  for (int mb = 0; mb < (ND == 2 ? 1 : Pm); ++mb) {
    const T wb = ND == 2 ? T(1) : a.mortar->I[mb][pb];
    for (int ma = 0; ma < Pm; ++ma) {
      const T w = a.mortar->I[ma][pa] * wb;
      const int tm = orient_inv(r.orient, ma + Pm * mb, Pm, ND);
      for (int c = 0; c < NC; ++c) acc[c] += w * sc[c * NFPm + tm];
    }
  }
  T* ts = a.trbar + r.st;
  const T* fbs = a.fbar + r.so;
  for (int v = 0; v < NV; ++v) {
    T x = acc[v];
    if (VISC) x -= fbs[(NV + v) * NFPs + pt];
    ts[v * NFPs + pt] = x;
  }
  if (VISC) {
    T Gb[ND][NV], dqb[ND][NV];
    for (int j = 0; j < ND; ++j)
      for (int v = 0; v < NV; ++v) Gb[j][v] = acc[NV + j * NV + v];
    gradient_to_ref_adjoint<ND>(a.geo_s, r.se, r.sf, pt, Gb, dqb);
    for (int d = 0; d < ND; ++d)
      for (int v = 0; v < NV; ++v) ts[(NV + d * NV + v) * NFPs + pt] = dqb[d][v];
  }
}

// Boundary faces adjoint.
template <typename T>
struct BndAdjArgs {
  const BndRec* recs;
  const T* trq;
  const T* fbar;
  T* trbar;
  const BasisTab<T>* basis;
  GeoView<T> geo;
  T gamma, mu, kappa;
  T qinf[5];
  int n, P, kind;
  int flux;            // common inviscid flux: 0 Rusanov, 1 Roe
};

template <typename T, int ND, bool VISC>
__global__ void __launch_bounds__(128) bnd_adj_kernel(BndAdjArgs<T> a) {
  constexpr int NV = ND + 2;
  const int P = a.P;
  const int NFP = ND == 2 ? P : P * P;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)a.n * NFP) return;
  const int t = (int)(gid % NFP);
  const BndRec r = a.recs[gid / NFP];
  const int d = r.mf >> 1, s = r.mf & 1;
  T qM[NV], qG[NV];
  load_trace_pt<ND>(a.trq, (const T*)nullptr, r.mt, 0, NV, NFP, t, qM);
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
  T Fnb[NV], qcb[NV], qMb[NV], qGb[NV];
  const T* fbm = a.fbar + r.mo;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Fnb[v] = sg * fbm[v * NFP + t];
    qcb[v] = VISC ? fbm[(NV + v) * NFP + t] : T(0);
    qMb[v] = VISC ? -fbm[(NV + v) * NFP + t] : T(0);
    qGb[v] = T(0);
  }
  flux_adjoint<ND>(a.flux, qM, qG, n, absA, a.gamma, Fnb, qMb, qGb);
  T GMb[ND][NV];
  if (VISC) {
    T qc[NV], cM[ND];
#pragma unroll
    for (int v = 0; v < NV; ++v) qc[v] = T(0.5) * (qM[v] + qG[v]);
    const T gJ = a.basis[P].dgf[s] * geo_face(a.geo, r.me, r.mf, ND * ND + 1, t);
#pragma unroll
    for (int j = 0; j < ND; ++j) cM[j] = gJ * geo_face(a.geo, r.me, r.mf, d * ND + j, t);
    T GM[ND][NV], Gc[ND][NV];
    load_trace_pt<ND>(a.trq, (const T*)nullptr, r.mt, NV, ND * NV, NFP, t, &GM[0][0]);
#pragma unroll
    for (int j = 0; j < ND; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) Gc[j][v] = GM[j][v] + cM[j] * (qc[v] - qM[v]);
    T fvb[ND][NV], Gcb[ND][NV], nfvb[ND][NV];
#pragma unroll
    for (int j = 0; j < ND; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        fvb[j][v] = (a.kind == -1 && v == NV - 1) ? T(0) : -Fnb[v] * A[j];
        nfvb[j][v] = -fvb[j][v];
      }
    viscous_adjoint_G<ND>(qc, fvb, a.gamma, a.mu, a.kappa, Gcb);
    flux_adjoint_q<ND>(qc, Gc, nfvb, a.gamma, a.mu, a.kappa, false, true, qcb);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T sM = T(0);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        GMb[j][v] = Gcb[j][v];
        sM += cM[j] * Gcb[j][v];
      }
      qcb[v] += sM;
      qMb[v] -= sM;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      qMb[v] += T(0.5) * qcb[v];
      qGb[v] += T(0.5) * qcb[v];
    }
  }
  // ghost-state transpose: wall reverses momentum; the far-field state is constant
  if (a.kind == -1) {
    qMb[0] += qGb[0];
#pragma unroll
    for (int i = 0; i < ND; ++i) qMb[1 + i] -= qGb[1 + i];
    qMb[NV - 1] += qGb[NV - 1];
  }
  T* tm = a.trbar + r.mt;
#pragma unroll
  for (int v = 0; v < NV; ++v) tm[v * NFP + t] = qMb[v];
  if (VISC) {
    T dqb[ND][NV];
    gradient_to_ref_adjoint<ND>(a.geo, r.me, r.mf, t, GMb, dqb);
#pragma unroll
    for (int dd = 0; dd < ND; ++dd)
#pragma unroll
      for (int v = 0; v < NV; ++v) tm[(NV + dd * NV + v) * NFP + t] = dqb[dd][v];
  }
}

// ---------------------------------------------------------------------------
// Trace adjoint: gather every face-point adjoint that depends on a solution
// point and add it to the volume part.  One thread per (element, sp).
// ---------------------------------------------------------------------------
template <typename T>
struct TraceAdjArgs {
  const T* trbar;
  T* out;              // in: volume part; out: full q-bar
  const BasisTab<T>* basis;
  int64_t state_base, trace_base;
  int count, nvt;
};

template <typename T, int ND, int P, bool VISC>
__global__ void __launch_bounds__(256) trace_adj_kernel(TraceAdjArgs<T> a) {
  using Sh = Shape<ND, P>;
  constexpr int NV = Sh::NV, NF = Sh::NF, NSP = Sh::NSP, NFP = Sh::NFP;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)a.count * NSP) return;
  const int sp = (int)(gid % NSP);
  const int64_t i = gid / NSP;
  const BasisTab<T>& B = a.basis[P];
  int idx[3];
  idx[0] = sp % P;
  idx[1] = (sp / P) % P;
  idx[2] = ND == 3 ? sp / (P * P) : 0;
  const T* tb = a.trbar + a.trace_base + i * NF * (int64_t)a.nvt * NFP;
  T acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = a.out[a.state_base + (i * NV + v) * NSP + sp];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const int tf = face_pt<ND, P>(d, idx);
    // tangential axes of face d and this point's coordinates on them
    const int ta = ND == 2 ? (d == 0 ? 1 : 0) : (d == 0 ? 1 : 0);
    const int tbx = ND == 2 ? -1 : (d == 2 ? 1 : 2);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T* blk = tb + (2 * d + s) * (int64_t)a.nvt * NFP;
      const T e = B.ext[s][idx[d]];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T x = e * blk[v * NFP + tf];
        if (VISC) {
          x += B.dext[s][idx[d]] * blk[(NV + d * NV + v) * NFP + tf];
          // tangential derivative adjoints along axis ta (first) and tbx (second)
#pragma unroll
          for (int c = 0; c < P; ++c) {
            const int t1 = ND == 2 ? c : (c + P * idx[tbx]);
            x += e * B.D[c][idx[ta]] * blk[(NV + ta * NV + v) * NFP + t1];
            if (ND == 3) {
              const int t2 = idx[ta] + P * c;
              x += e * B.D[c][idx[tbx]] * blk[(NV + tbx * NV + v) * NFP + t2];
            }
          }
        }
        acc[v] += x;
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) a.out[a.state_base + (i * NV + v) * NSP + sp] = acc[v];
}

}  // namespace frgb
