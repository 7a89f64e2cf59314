// Pointwise physics of the compressible Navier-Stokes equations (Sec. 2.1),
// written once over a scalar type S: S = T gives the residual, S = Dual<T>
// (value + directional derivative) gives the exact JVP by forward-mode
// differentiation of the same arithmetic.
#pragma once

#include <cuda_runtime.h>

#include "dfloat.cuh"

namespace frgb {

template <typename T>
struct Dual {
  T v, d;
};

template <typename T>
__device__ __forceinline__ T value(T x) { return x; }
template <typename T>
__device__ __forceinline__ T value(Dual<T> x) { return x.v; }
template <typename T>
__device__ __forceinline__ T tangent(T) { return T(0); }
template <typename T>
__device__ __forceinline__ T tangent(Dual<T> x) { return x.d; }

template <typename T>
__device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T r = a.v / b.v;
  return {r, (a.d - r * b.d) / b.v};
}
template <typename T>
__device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator+(T a, Dual<T> b) { return {a + b.v, b.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return {a.v - b, a.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return {a - b.v, -b.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator/(Dual<T> a, T b) { return {a.v / b, a.d / b}; }
template <typename T>
__device__ __forceinline__ Dual<T> operator/(T a, Dual<T> b) {
  T r = a / b.v;
  return {r, -r * b.d / b.v};
}

// acc + a * b: one FMA in FP64/FP32 (the compiler contracts it), one fused
// double-float operation for dfloat
template <typename S, typename A, typename B>
__device__ __forceinline__ S madd(S acc, A a, B b) { return acc + a * b; }
__device__ __forceinline__ dfloat madd(dfloat acc, dfloat a, dfloat b) { return dfma(a, b, acc); }

// Accumulator of a short contraction c + sum_k a_k b_k: the plain type for
// FP64, FP32 and dual numbers; for double-float an unnormalised pair whose
// high part is summed exactly (TwoSum) and whose error terms are summed in
// FP32, normalised once at the end (12 FP32 operations a term instead of 15;
// the FP32 sum of the error terms adds about n u^2 sum_k |a_k b_k|).
template <typename S>
struct Acc {
  S v;
};
template <typename S>
__device__ __forceinline__ Acc<S> acc_init(S x) { return Acc<S>{x}; }
template <typename S, typename A, typename B>
__device__ __forceinline__ void acc_madd(Acc<S>& c, A a, B b) { c.v = madd(c.v, a, b); }
template <typename S>
__device__ __forceinline__ S acc_value(const Acc<S>& c) { return c.v; }

template <>
struct Acc<dfloat> {
  float s, e;
};
__device__ __forceinline__ Acc<dfloat> acc_init(dfloat x) { return Acc<dfloat>{x.hi, x.lo}; }
__device__ __forceinline__ void acc_madd(Acc<dfloat>& c, dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  float s, t;
  dfl::two_sum(c.s, p, s, t);
  c.s = s;
  c.e = __fadd_rn(c.e, __fadd_rn(t, pe));
}
__device__ __forceinline__ dfloat acc_value(const Acc<dfloat>& c) { return dfl::renorm(c.s, c.e); }

__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
template <typename T>
__device__ __forceinline__ Dual<T> dsqrt(Dual<T> x) {
  T r = dsqrt(x.v);
  return {r, x.d / (T(2) * r)};
}
// |x| with d|x| = sign(x) dx, sign(0) := +1
__device__ __forceinline__ double dabs(double x) { return fabs(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }
template <typename T>
__device__ __forceinline__ Dual<T> dabs(Dual<T> x) { return x.v < T(0) ? Dual<T>{-x.v, -x.d} : x; }
// max(a, b); at a tie the first argument (the "-" side) is taken
template <typename T>
__device__ __forceinline__ T dmax(T a, T b) { return b > a ? b : a; }
template <typename T>
__device__ __forceinline__ Dual<T> dmax(Dual<T> a, Dual<T> b) { return b.v > a.v ? b : a; }

template <typename S>
__device__ __forceinline__ S szero() { return S{}; }

template <typename T>
__device__ __forceinline__ void set_scalar(T& x, T v, T) { x = v; }
template <typename T>
__device__ __forceinline__ void set_scalar(Dual<T>& x, T v, T d) { x.v = v; x.d = d; }

// Inviscid flux f[j][v] (physical direction j) of q = (rho, rho u_i, rho E).
template <int ND, typename S, typename T>
__device__ __forceinline__ void flux_inviscid(const S* q, T gamma, S (*f)[ND + 2]) {
  constexpr int NV = ND + 2;
  const S rinv = T(1) / q[0];
  S vel[ND];
  S mu2 = szero<S>();
#pragma unroll
  for (int i = 0; i < ND; ++i) vel[i] = q[1 + i] * rinv;
#pragma unroll
  for (int i = 0; i < ND; ++i) mu2 = mu2 + q[1 + i] * vel[i];
  const S pres = (gamma - T(1)) * (q[NV - 1] - T(0.5) * mu2);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    f[j][0] = q[1 + j];
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      S fij = q[1 + i] * vel[j];
      if (i == j) fij = fij + pres;
      f[j][1 + i] = fij;
    }
    f[j][NV - 1] = (q[NV - 1] + pres) * vel[j];
  }
}

// Normal flux f(q).n and the wave speed |u.n| + c of one state (one reciprocal,
// one square root).
template <int ND, typename S, typename T>
__device__ __forceinline__ S normal_flux(const S* q, const T* n, T gamma, S* fn) {
  constexpr int NV = ND + 2;
  const S rinv = T(1) / q[0];
  S mn = szero<S>(), mu2 = szero<S>();
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    mn = mn + q[1 + i] * n[i];
    mu2 = mu2 + q[1 + i] * q[1 + i];
  }
  const S un = mn * rinv;
  const S pres = (gamma - T(1)) * (q[NV - 1] - T(0.5) * mu2 * rinv);
  fn[0] = mn;
#pragma unroll
  for (int i = 0; i < ND; ++i) fn[1 + i] = q[1 + i] * un + pres * n[i];
  fn[NV - 1] = (q[NV - 1] + pres) * un;
  return dabs(un) + dsqrt(gamma * pres * rinv);
}

// Normal flux f(q).n alone (no wave speed).
template <int ND, typename S, typename T>
__device__ __forceinline__ void normal_flux_only(const S* q, const T* n, T gamma, S* fn) {
  constexpr int NV = ND + 2;
  const S rinv = T(1) / q[0];
  S mn = szero<S>(), mu2 = szero<S>();
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    mn = mn + q[1 + i] * n[i];
    mu2 = mu2 + q[1 + i] * q[1 + i];
  }
  const S un = mn * rinv;
  const S pres = (gamma - T(1)) * (q[NV - 1] - T(0.5) * mu2 * rinv);
  fn[0] = mn;
#pragma unroll
  for (int i = 0; i < ND; ++i) fn[1 + i] = q[1 + i] * un + pres * n[i];
  fn[NV - 1] = (q[NV - 1] + pres) * un;
}

// Roe's flux times the face area: ((fL.n + fR.n)/2 - |A| (qR - qL)/2) |A_f|,
// |A| the absolute normal flux Jacobian at Roe's averages (sqrt(rho)-weighted
// velocity and total enthalpy), applied through the closed-form wave
// strengths of the acoustic (u.n -+ c), entropy and shear (u.n) waves instead
// of the eigenvector matrices.  No entropy fix; |x| via dabs (sign(0) = +1).
template <int ND, typename S, typename T>
__device__ __forceinline__ void roe(const S* qL, const S* qR, const T* n, T absA, T gamma, S* Fn) {
  constexpr int NV = ND + 2;
  S fL[NV], fR[NV];
  normal_flux_only<ND>(qL, n, gamma, fL);
  normal_flux_only<ND>(qR, n, gamma, fR);
  const S riL = T(1) / qL[0], riR = T(1) / qR[0];
  S uL[ND], uR[ND], kL = szero<S>(), kR = szero<S>();
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    uL[i] = qL[1 + i] * riL;
    uR[i] = qR[1 + i] * riR;
    kL = kL + qL[1 + i] * uL[i];
    kR = kR + qR[1 + i] * uR[i];
  }
  const S pL = (gamma - T(1)) * (qL[NV - 1] - T(0.5) * kL);
  const S pR = (gamma - T(1)) * (qR[NV - 1] - T(0.5) * kR);
  const S HL = (qL[NV - 1] + pL) * riL, HR = (qR[NV - 1] + pR) * riR;
  const S sL = dsqrt(qL[0]), sR = dsqrt(qR[0]);
  const S wi = T(1) / (sL + sR);
  S u[ND], q2 = szero<S>(), un = szero<S>(), dun = szero<S>(), udu = szero<S>();
  S du[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    u[i] = (sL * uL[i] + sR * uR[i]) * wi;
    du[i] = uR[i] - uL[i];
    q2 = q2 + u[i] * u[i];
    un = un + u[i] * n[i];
    dun = dun + du[i] * n[i];
    udu = udu + u[i] * du[i];
  }
  const S H = (sL * HL + sR * HR) * wi;
  const S c2 = (gamma - T(1)) * (H - T(0.5) * q2);
  const S c = dsqrt(c2);
  const S rho = sL * sR;
  const S dp = pR - pL, drho = qR[0] - qL[0];
  const S ic2 = T(1) / c2;
  const S a1 = T(0.5) * (dp - rho * c * dun) * ic2;
  const S a3 = T(0.5) * (dp + rho * c * dun) * ic2;
  const S a2 = drho - dp * ic2;
  const S l1 = dabs(un - c) * a1, l2 = dabs(un), l3 = dabs(un + c) * a3;
  S d[NV];
  d[0] = l1 + l2 * a2 + l3;
#pragma unroll
  for (int i = 0; i < ND; ++i)
    d[1 + i] = l1 * (u[i] - c * n[i]) + l2 * (a2 * u[i] + rho * (du[i] - dun * n[i])) + l3 * (u[i] + c * n[i]);
  d[NV - 1] = l1 * (H - c * un) + l2 * (a2 * T(0.5) * q2 + rho * (udu - un * dun)) + l3 * (H + c * un);
#pragma unroll
  for (int v = 0; v < NV; ++v) Fn[v] = (T(0.5) * (fL[v] + fR[v]) - T(0.5) * d[v]) * absA;
}

// Rusanov normal flux times the face area: ((fL.n + fR.n)/2 - lam/2 (qR - qL)) |A|,
// lam = max(|u.n| + c) over the two sides (the "-" side at a tie).
template <int ND, typename S, typename T>
__device__ __forceinline__ void rusanov(const S* qL, const S* qR, const T* n, T absA, T gamma,
                                        S* Fn) {
  constexpr int NV = ND + 2;
  S fL[NV], fR[NV];
  const S lamL = normal_flux<ND>(qL, n, gamma, fL);
  const S lamR = normal_flux<ND>(qR, n, gamma, fR);
  const S lam = dmax(lamL, lamR);
#pragma unroll
  for (int v = 0; v < NV; ++v) Fn[v] = (T(0.5) * (fL[v] + fR[v]) - T(0.5) * lam * (qR[v] - qL[v])) * absA;
}

// The common inviscid flux of a face: Rusanov (kind 0) or Roe (kind 1).
template <int ND, typename S, typename T>
__device__ __forceinline__ void common_flux(int kind, const S* qL, const S* qR, const T* n, T absA, T gamma,
                                            S* Fn) {
  if (kind == 1) roe<ND>(qL, qR, n, absA, gamma, Fn);
  else rusanov<ND>(qL, qR, n, absA, gamma, Fn);
}

// Viscous flux fv[j][v] from q and its physical gradient G[j][v]:
// (0, tau_ij, u_i tau_ij + kappa d_j(p/rho)), kappa = mu gamma / ((gamma-1) Pr).
template <int ND, typename S, typename T>
__device__ __forceinline__ void flux_viscous(const S* q, const S (*G)[ND + 2], T gamma, T mu,
                                             T kappa, S (*fv)[ND + 2]) {
  constexpr int NV = ND + 2;
  const S rinv = T(1) / q[0];
  S vel[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) vel[i] = q[1 + i] * rinv;
  const S Es = q[NV - 1] * rinv;
  S du[ND][ND];
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) du[i][j] = (G[j][1 + i] - vel[i] * G[j][0]) * rinv;
  S dT[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    S dE = (G[j][NV - 1] - Es * G[j][0]) * rinv;
    S s = szero<S>();
#pragma unroll
    for (int k = 0; k < ND; ++k) s = s + vel[k] * du[k][j];
    dT[j] = (gamma - T(1)) * (dE - s);
  }
  S div = szero<S>();
#pragma unroll
  for (int k = 0; k < ND; ++k) div = div + du[k][k];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    fv[j][0] = szero<S>();
    S e = szero<S>();
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      S tau = mu * (du[i][j] + du[j][i]);
      if (i == j) tau = tau - T(2.0 / 3.0) * mu * div;
      fv[j][1 + i] = tau;
      e = e + vel[i] * tau;
    }
    fv[j][NV - 1] = e + kappa * dT[j];
  }
}

// Row d of the viscous flux, fv[d][v] (the flux through a face normal to axis
// d): the same arithmetic as flux_viscous restricted to that row.
template <int ND, typename S, typename T>
__device__ __forceinline__ void flux_viscous_row(const S* q, const S (*G)[ND + 2], T gamma, T mu, T kappa,
                                                 int d, S* fr) {
  constexpr int NV = ND + 2;
  const S rinv = T(1) / q[0];
  S vel[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) vel[i] = q[1 + i] * rinv;
  const S Es = q[NV - 1] * rinv;
  S du[ND][ND];
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) du[i][j] = (G[j][1 + i] - vel[i] * G[j][0]) * rinv;
  S div = szero<S>();
#pragma unroll
  for (int k = 0; k < ND; ++k) div = div + du[k][k];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    if (j != d) continue;
    S dE = (G[j][NV - 1] - Es * G[j][0]) * rinv;
    S s = szero<S>();
#pragma unroll
    for (int k = 0; k < ND; ++k) s = s + vel[k] * du[k][j];
    const S dT = (gamma - T(1)) * (dE - s);
    fr[0] = szero<S>();
    S e = szero<S>();
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      S tau = mu * (du[i][j] + du[j][i]);
      if (i == j) tau = tau - T(2.0 / 3.0) * mu * div;
      fr[1 + i] = tau;
      e = e + vel[i] * tau;
    }
    fr[NV - 1] = e + kappa * dT;
  }
}

// Ghost state of a boundary: wall (-1) reverses momentum, far field (-2) is q_inf.
template <int ND, typename S, typename T>
__device__ __forceinline__ void ghost_state(const S* q, int kind, const T* qinf, S* g) {
  constexpr int NV = ND + 2;
  if (kind == -1) {
    g[0] = q[0];
#pragma unroll
    for (int i = 0; i < ND; ++i) g[1 + i] = -q[1 + i];
    g[NV - 1] = q[NV - 1];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) set_scalar(g[v], qinf[v], T(0));
  }
}

}  // namespace frgb
